// K2: the fused domain-selection step (Sec. III-B) for dense J on the
// tcgen05 tensor cores.
//
// G = J S is a GEMM with M = spins (J rows, 128 per tile), N = restarts (BN
// per tile) and K = spins. J is stored as E4M3 [n][ld] when every J is an
// integer of magnitude <= 16 (exact), as one BF16 plane when every J is an
// integer of magnitude <= 256 (exact), else as FP16 planes: one for integers
// up to 2048, hi + lo for integers up to 65504 (both exact) and for other J,
// which are first divided by a power-of-two scale per row (about 22
// significant bits; the epilogue multiplies the row's product back, exactly).
// The spins S_t are +-1 of the same type [B][ld] (restart-major, K
// contiguous; kind::f16 takes both operands in one type). Both operands are
// K-major, so one TMA box of 128 bytes (a k-block: 128 E4M3 or 64 16-bit
// elements) x rows fills a 128-byte swizzled shared-memory tile that
// tcgen05.mma reads directly. A thread issues one tcgen05.mma only every ~110
// cycles and one TMA copy every ~250 whatever their sizes, which shapes the
// kernels below.
//
// Streaming form (tc_step_kernel): one persistent CTA per SM, warp-specialised:
//   warps 0, 2 TMA producers of the J and the S tiles of a STAGES-deep ring
//              (stages of two k-blocks for BN <= 128, of one for BN = 256;
//              with two J planes a stage is one k-block of both planes and
//              its spin tile, and the MMAs take the planes k-block by
//              k-block, the order every form uses),
//   warp 1     allocates tensor memory and issues the MMAs (one thread) into
//              one of two accumulator buffers (2 x BN columns of 128 lanes),
//   warps 4-19 epilogue: each thread owns one spin i (its TMEM lane) and walks
//              a quarter of the tile's restarts 8 columns at a time (the chunk's
//              state is loaded into registers while the TMEM read lands): loss field
//              F = cQ G + cH h - mu s, gradient cos(theta) F, Adam, projection,
//              new spin into S_{t+1}, and the energy of the input spins, summed
//              over each warp's 32 spins by a butterfly across lanes into
//              one partial row per warp (summed in fixed order afterwards).
// The same roles run in clusters of two CTAs (tc_step_pair_kernel: each
// loads half of the spin tile and multicasts it to both; tc_step_split_kernel:
// the pair's MMAs issued as one, cta_group::2, M 256, each CTA holding its J
// rows and half of the spin tile), shapes the autotuner times beside single
// CTAs.
// Tiles are numbered row tile by row tile (the restart tiles of one row tile
// are consecutive), so one wave of persistent CTAs covers whole row tiles: a
// J row tile is read from HBM about once per step and shared through L2 by
// the CTAs of its wave, and only the (smaller) spin operand is read by every
// wave.
// While the epilogue drains one accumulator the MMA fills the other. Every
// mbarrier wait is bounded; a timeout sets an error word and the CTA drains
// its in-flight copies and MMAs, frees tensor memory and returns.
#include "ds_internal.cuh"
#include "tcgen05.cuh"

#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include <algorithm>

namespace ising {
namespace {

constexpr int kBM = 128;
constexpr int kRowBytes = 128;  // one 128-byte swizzled row per operand row and k-block
constexpr int kEpiWarps = 16;  // four per TMEM lane quarter, each owning a quarter of the columns
constexpr int kChunk = 8;      // columns per TMEM read
constexpr int kThreads = 128 + 32 * kEpiWarps;
constexpr long long kWaitCycles = 4000000000ll;  // about 2 s

struct TcArgs {
  int64_t n, B, ld;
  int nk;      // k-blocks per plane
  int planes;  // 1 or 2
  int f16;     // 16-bit operands are FP16 (else BF16): MMA input format and spin encoding
  int mtiles, ntiles;
  StepConsts k;
  const float2* bias;
  const long long* counters;
  const void* S;           // S_t, [B][ld] (BF16 or E4M3)
  void* Snext;             // S_{t+1}
  void* Xnext;             // relaxed mode: x_{t+1} = sin(theta), BF16 [B][ld]
  const float* rowscale;   // FP8 path with scaled rows, else null
  float* theta;
  float* m;
  float* v;
  const float* hf;
  const int32_t* hint;
  long long* qpart;
  long long* hpart;
  float* epart;
  float* Gout;  // coupling mode: [B][ld]
  int* err;
  int has_h;
  int gmagic;  // resident epilogue's integer energy mode (EMODE of resident_chunks)
  unsigned long long* trace;  // per-CTA role timeline (profiling), or null
  int nfull;   // streaming kernel: whole k-blocks loadable in pairs (0: never pair)
  const int* live32;          // convergence rule: live restarts per 32 (tiles retire), or null
  unsigned long long* work;   // restart-steps computed (update launches), or null
  // update launches of one instance: track the step before this one (the
  // epilogue warps, while the first tile's products run) and advance the
  // step counter at the end, instead of a tracking launch after each step
  int fold = 0;
  TrackArgs trk;
};

// +1 / -1 in the 16-bit operand type (FP16 0x3C00, BF16 0x3F80; bit 15 is the
// sign in both, so readers of either test that bit).
__device__ __forceinline__ uint16_t pm1_16(bool pos, int f16) {
  return (uint16_t)((f16 ? 0x3C00u : 0x3F80u) | (pos ? 0u : 0x8000u));
}

// x rounded to nearest in the 16-bit operand type, as its bit pattern.
__device__ __forceinline__ uint16_t to_op16(float x, int f16) {
  return f16 ? __half_as_ushort(__float2half_rn(x)) : __bfloat16_as_ushort(__float2bfloat16(x));
}

// Instruction descriptor of an M x N tile (M 128, or 256 for a CTA pair):
// kind::f8f6f4 E4M3 (format 0), or kind::f16 with FP16 (format 0) or BF16
// (format 1) inputs.
__device__ __forceinline__ uint32_t op_idesc(int N, bool fp8, int f16, int M = 128) {
  return tc::idesc_make(M, N, fp8 ? 0u : (f16 ? 0u : 1u));
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t)::"memory");
  return t;
}

// Trace slots per CTA (globaltimer, ns): 0 start, 1 first TMA issued, 2 last
// TMA issued, 3 first MMA issued, 4 last MMA committed, 5 epilogue has its
// first accumulator, 6 epilogue done (warp 4), 7 end.

// Streaming form: for BN <= 128 stages of two k-blocks [J, J, S, S], so that
// two whole k-blocks of one plane arrive by one copy per operand (a thread
// issues one TMA copy per ~250 cycles whatever its size); for BN = 224 and
// 256 such stages would leave room for two only, so there a stage is one
// k-block.
// With two J planes a stage instead holds one k-block of both planes and the
// spin tile of that k-block, which both planes' MMAs read (a third less to
// copy and to store per MMA than a stage per plane and k-block).
template <int BN, bool SPLIT = false>
struct TcLayout {
  static constexpr int kKps = BN >= 192 ? 1 : 2;
  static constexpr uint32_t kA = kBM * kRowBytes;
  // SPLIT (the MMA of a CTA pair): each CTA holds half of the spin tile
  static constexpr uint32_t kB = (SPLIT ? BN / 2 : BN) * kRowBytes;
  static constexpr uint32_t kStage = kKps * (kA + kB);
  static constexpr uint32_t kStage2 = 2 * kA + kB;  // two planes
  // SPLIT: a spin half's worth of room after the last stage, so that every
  // operand read of a stage stays inside this CTA's shared memory whatever
  // part of the pair's tile it covers
  static constexpr uint32_t kTail = SPLIT ? kB : 0;
  // as many stages as the 225 KB region holds (the ring's depth covers the
  // latency of the operand copies from L2), then the barrier block
  static constexpr uint32_t kRegion = 225 * 1024;
  static constexpr uint32_t kBytes = kRegion + 256 + 1024;  // + alignment slack
  // two accumulator buffers; allocations are powers of two columns
  static constexpr uint32_t kTmemCols = 2 * BN <= 128 ? 128 : (2 * BN <= 256 ? 256 : 512);
};

// Resident form: shared memory holds the first `jres` J tiles of the CTA's
// rows for the whole run (J does not change between steps), then `nst`
// stages of a J tile and the S tile of one restart group (GN); the later J
// tiles stream through the stages. Sizes are chosen at launch (TcResArgs).
template <int GN>
struct ResLayout {
  static constexpr int kKps = 2;  // k-blocks per stage: [J tiles][S tiles]
  static constexpr uint32_t kA = kBM * kRowBytes;
  static constexpr uint32_t kB = GN * kRowBytes;
  static constexpr uint32_t kStage = kKps * (kA + kB);
  static constexpr int kMaxStages = 8;
};

// Sum over the 32 lanes of each of 8 columns; afterwards lanes l, l^1, l^2,
// l^3 hold the total of column 4 b4 + 2 b3 + b2 (bits of l).
template <typename T>
__device__ __forceinline__ T column_sums8(T (&x)[8], int lane) {
#pragma unroll
  for (int o = 16, len = 4; o >= 4; o >>= 1, len >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < len; ++j) {
      T send = up ? x[j] : x[j + len];
      T keep = up ? x[j + len] : x[j];
      x[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  T y = x[0] + __shfl_xor_sync(0xffffffffu, x[0], 2);
  return y + __shfl_xor_sync(0xffffffffu, y, 1);
}

__device__ __forceinline__ int column_of_lane(int lane) {
  return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}

// One tile of a step launch: the instance it belongs to (its arguments, the
// operand maps, the spin and partial slots of its current step) and where
// the tile lies (row tile mt, first row m0, first restart n0).
struct TileRef {
  const TcArgs* P;
  const CUtensorMap *A0, *A1, *A2;  // J planes, boxes of one k-block
  const CUtensorMap *J0, *J1, *J2;  // J planes, boxes of two k-blocks
  const CUtensorMap* B;      // S_t, boxes of one k-block x BN restarts
  const CUtensorMap* S2;     // S_t, boxes of two k-blocks
  const void* S;             // S_t
  void* Snext;               // S_{t+1}
  long long* qpart;
  long long* hpart;
  float* epart;
  int mt, m0, n0;
  bool skip;  // every restart of the tile has stopped (convergence rule)
  __device__ const CUtensorMap* a(int plane) const { return plane == 0 ? A0 : (plane == 1 ? A1 : A2); }
  __device__ const CUtensorMap* j2(int plane) const { return plane == 0 ? J0 : (plane == 1 ? J1 : J2); }
};

// Called by every CTA of a launch at its end: `done` counts the CTAs that
// got here, and the last one (every CTA has read the step counters by then)
// resets it and, for the session (`ctr`) or each of `count` pack members
// (trk[e].counters), records the step before this launch's as tracked
// ([2]) and adds one to the step counter ([0]).
__device__ __forceinline__ void advance_counters(unsigned long long* done, long long* ctr,
                                                 const TrackArgs* trk, int count) {
  if (threadIdx.x != 0) return;
  __threadfence();
  if (atomicAdd(done, 1ull) != gridDim.x - 1) return;
  for (int e = 0; e < (trk ? count : 1); ++e) {
    long long* c = trk ? trk[e].counters : ctr;
    if (c[0] > c[2]) c[2] = c[0];
    c[0] += 1;
  }
  *done = 0;
  __threadfence();
}

// Tiles of one instance: everything comes from the kernel's parameters (the
// host chose the slots of step t), tiles numbered row tile by row tile.
template <int BN>
struct OneInstance {
  static constexpr bool kGlobalMaps = false;  // kernel parameters
  static constexpr bool kPair = false;
  static constexpr bool kSplit = false;
  static constexpr bool kFold = true;  // may track the previous step (TcArgs::fold)
  const TcArgs& P;  // the kernel's parameter
  const CUtensorMap *A0, *A1, *A2, *B, *J0, *J1, *J2, *S2;
  __device__ int first() const { return blockIdx.x; }
  __device__ int stride() const { return gridDim.x; }
  // the CTA's j-th tile
  __device__ int at(int j) const { return first() + j * stride(); }
  __device__ int total() const { return P.mtiles * P.ntiles; }
  __device__ int* err() const { return P.err; }
  __device__ unsigned long long* trace() const { return P.trace; }
  __device__ bool fused() const { return P.planes == 2; }
  // (update launches with P.fold) the previous step's tracking, by warp gw
  // of nw, and the counter advance by the last CTA
  template <int KIND>
  __device__ void track_prev(int64_t gw, int64_t nw, int lane) const {
    const long long tp = P.counters[0];
    if (!P.fold || tp < 1 || tp <= P.counters[2]) return;  // none, or already tracked
    for (int64_t b = gw; b < P.trk.B; b += nw) track_restart<KIND>(P.trk, tp, b, lane);
  }
  __device__ void advance_step() const {
    if (P.fold)
      advance_counters(reinterpret_cast<unsigned long long*>(&P.trk.counters[1]), P.trk.counters,
                       nullptr, 0);
  }
  __device__ const TcArgs& args(const TileRef&) const { return P; }
  __device__ TileRef tile(int tl) const {
    TileRef r;
    r.P = &P;
    r.A0 = A0; r.A1 = A1; r.A2 = A2;
    r.J0 = J0; r.J1 = J1; r.J2 = J2;
    r.B = B;
    r.S2 = S2;
    r.S = P.S;
    r.Snext = P.Snext;
    r.qpart = P.qpart;
    r.hpart = P.hpart;
    r.epart = P.epart;
    r.mt = tl / P.ntiles;
    r.m0 = r.mt * kBM;
    r.n0 = (tl % P.ntiles) * BN;
    r.skip = restarts_retired(P.live32, r.n0, min((int64_t)r.n0 + BN, P.B));
    return r;
  }
};

// One member of a packed launch (several instances advanced by one step in
// one launch): its arguments and maps in device memory, with all three spin
// slots and both partial slots; the slots of its step come from its own
// device step counter, so every launch of a pack is identical whatever the
// members' progress (the step loop can be replayed from a CUDA graph).
struct __align__(64) PackEntry {
  CUtensorMap A[3];
  CUtensorMap J2[3];
  CUtensorMap B[3];   // per spin slot
  CUtensorMap S2[3];  // per spin slot
  TcArgs args;
  void* spins[3];
  long long* qpart[2];
  long long* hpart[2];
  float* epart[2];
};

// Tiles of a pack: member e owns tiles [start[e], start[e + 1]).
template <int BN>
struct PackedInstances {
  static constexpr bool kGlobalMaps = true;  // copied to device memory by the host
  static constexpr bool kPair = false;
  static constexpr bool kSplit = false;
  static constexpr bool kFold = true;  // may track every member's previous step (trk)
  __device__ int first() const { return blockIdx.x; }
  __device__ int stride() const { return gridDim.x; }
  // the CTA's j-th tile: the tiles are taken wave by wave (a wave is one
  // tile per CTA), every other wave in reverse CTA order, so that over the
  // waves of a pack sorted by tile size no CTA draws the largest tile of
  // each wave
  __device__ int at(int j) const {
    const int g = gridDim.x, c = blockIdx.x;
    return j * g + ((j & 1) ? g - 1 - c : c);
  }
  const PackEntry* E;
  const int* start;
  int count;
  int* errp;
  bool planes2;  // every member has two J planes (members share the count)
  // the members' tracking arguments and restart offsets when the launch
  // tracks every member's previous step (else null)
  const TrackArgs* trk;
  const int64_t* rstart;
  unsigned long long* done;  // the pack's CTA counter
  __device__ int total() const { return start[count]; }
  __device__ int* err() const { return errp; }
  __device__ unsigned long long* trace() const { return nullptr; }
  __device__ bool fused() const { return planes2; }
  template <int KIND>
  __device__ void track_prev(int64_t gw, int64_t nw, int lane) const {
    if (!trk) return;
    for (int64_t g = gw; g < rstart[count]; g += nw) {
      int lo = 0, hi = count - 1;
      while (lo < hi) {  // last member whose first restart is <= g
        const int mid = (lo + hi + 1) >> 1;
        if (rstart[mid] <= g) lo = mid; else hi = mid - 1;
      }
      const TrackArgs& A = trk[lo];
      const long long tp = A.counters[0];
      if (tp >= 1 && tp > A.counters[2]) track_restart<KIND>(A, tp, g - rstart[lo], lane);
    }
  }
  __device__ void advance_step() const {
    if (trk) advance_counters(done, nullptr, trk, count);
  }
  __device__ const TcArgs& args(const TileRef& T) const { return *T.P; }
  __device__ TileRef tile(int tl) const {
    int lo = 0, hi = count - 1;
    while (lo < hi) {  // last member whose first tile is <= tl
      const int mid = (lo + hi + 1) >> 1;
      if (start[mid] <= tl) lo = mid; else hi = mid - 1;
    }
    const PackEntry& e = E[lo];
    const long long t = e.args.counters[0] + 1;
    const int s0 = (int)(t % 3), s1 = (int)((t + 1) % 3), ps = (int)(t % 2);
    TileRef r;
    r.P = &e.args;
    r.A0 = &e.A[0]; r.A1 = &e.A[1]; r.A2 = &e.A[2];
    r.J0 = &e.J2[0]; r.J1 = &e.J2[1]; r.J2 = &e.J2[2];
    r.B = &e.B[s0];
    r.S2 = &e.S2[s0];
    r.S = e.spins[s0];
    r.Snext = e.spins[s1];
    r.qpart = e.qpart[ps];
    r.hpart = e.hpart[ps];
    r.epart = e.epart[ps];
    const int local = tl - start[lo];
    r.mt = local / e.args.ntiles;
    r.m0 = r.mt * kBM;
    r.n0 = (local % e.args.ntiles) * BN;
    r.skip = restarts_retired(e.args.live32, r.n0, min((int64_t)r.n0 + BN, e.args.B));
    return r;
  }
};

// Tiles of one instance for clusters of two CTAs: a cluster takes pair tile
// (pm, nt), its CTA of rank r the row tile 2 pm + r of restart tile nt. Both
// CTAs need the same spin tile: each loads one half of it and multicasts the
// half to both (the J tiles are their own), so a CTA reads 30 instead of 44
// KB per stage from L2 at tiles of 224 restarts. With an odd number of row
// tiles the last pair's second tile lies past n (zero rows, nothing written).
// SPLIT: instead of multicasting, each CTA keeps its half of the spin tile
// and the first CTA issues the MMAs of the pair (cta_group::2, M 256): a
// CTA's shared memory then holds and serves 30 instead of 44 KB per stage,
// which is what limits the operand stream of single-CTA tiles (the tensor
// cores read a stage as fast as TMA writes it, both through the SM's shared
// memory).
template <int BN, bool SPLIT = false>
struct PairInstance {
  static constexpr bool kGlobalMaps = false;
  static constexpr bool kPair = true;
  static constexpr bool kSplit = SPLIT;
  static constexpr bool kFold = true;
  const TcArgs& P;
  const CUtensorMap *A0, *A1, *A2, *B, *J0, *J1, *J2, *S2;
  const CUtensorMap* Bh;  // S_t, boxes of one k-block x BN / 2 restarts
  uint32_t rank;
  __device__ int first() const { return (int)tc::cluster_index(); }
  __device__ int stride() const { return (int)tc::cluster_count(); }
  // the CTA's j-th tile (row-tile-major order)
  __device__ int at(int j) const { return first() + j * stride(); }
  __device__ int total() const { return (P.mtiles + 1) / 2 * P.ntiles; }
  __device__ int* err() const { return P.err; }
  __device__ unsigned long long* trace() const { return P.trace; }
  __device__ bool fused() const { return P.planes == 2; }
  template <int KIND>
  __device__ void track_prev(int64_t gw, int64_t nw, int lane) const {
    const long long tp = P.counters[0];
    if (!P.fold || tp < 1 || tp <= P.counters[2]) return;  // none, or already tracked
    for (int64_t b = gw; b < P.trk.B; b += nw) track_restart<KIND>(P.trk, tp, b, lane);
  }
  __device__ void advance_step() const {
    if (P.fold)
      advance_counters(reinterpret_cast<unsigned long long*>(&P.trk.counters[1]), P.trk.counters,
                       nullptr, 0);
  }
  __device__ const TcArgs& args(const TileRef&) const { return P; }
  __device__ TileRef tile(int tl) const {
    TileRef r;
    r.P = &P;
    r.A0 = A0; r.A1 = A1; r.A2 = A2;
    r.J0 = J0; r.J1 = J1; r.J2 = J2;
    r.B = Bh;
    r.S2 = S2;
    r.S = P.S;
    r.Snext = P.Snext;
    r.qpart = P.qpart;
    r.hpart = P.hpart;
    r.epart = P.epart;
    r.mt = 2 * (tl / P.ntiles) + (int)rank;
    r.m0 = r.mt * kBM;
    r.n0 = (tl % P.ntiles) * BN;
    r.skip = restarts_retired(P.live32, r.n0, min((int64_t)r.n0 + BN, P.B));
    return r;
  }
};

#define ISING_TRACE(slot)                                                            \
  do {                                                                               \
    if (trace_) trace_[(size_t)blockIdx.x * 8 + (slot)] = now_ns();                  \
  } while (0)

// The persistent, warp-specialised step over the tiles of `src` (one
// instance, or the members of a pack). Roles as described at the top.
template <int BN, int MODE, bool INT_E, bool FP8, class Src>
__device__ __forceinline__ void step_tiles(const Src& src) {
  constexpr bool SPLIT = Src::kSplit;
  using Lay = TcLayout<BN, SPLIT>;
  constexpr int kBK = FP8 ? 128 : 64;  // elements per 128-byte row
  static_assert(!Src::kPair || Lay::kKps == 1, "pair tiles take one k-block per stage");
  // two J planes (every tile of the launch): stages of one k-block of both
  // planes and its spin tile, the MMAs taking the planes k-block by k-block
  const bool fused = !FP8 && src.fused();
  const uint32_t kSt = fused ? Lay::kStage2 : Lay::kStage;
  const int STAGES = (int)((Lay::kRegion - Lay::kTail) / kSt);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (uint32_t)STAGES * kSt + Lay::kTail);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  unsigned long long* const trace_ = src.trace();
  // SPLIT: the first CTA of the pair (rank 0) issues the MMAs of both
  bool lead = true;
  if constexpr (SPLIT) lead = src.rank == 0;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full[s], 2);  // the J and the S producer
      // released by the MMA issuer of each CTA of a multicasting pair, or by
      // the one issuer of a split pair (or of a single CTA)
      tc::mbar_init(&empty[s], (Src::kPair && !SPLIT) ? 2 : 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      // SPLIT: the first CTA's buffer is released by the epilogues of both
      tc::mbar_init(&acc_empty[b], SPLIT ? 2 * kEpiWarps : kEpiWarps);
    }
    tc::mbar_init(drain, 1);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) {
    if constexpr (SPLIT) tc::tmem_alloc_pair(tmem_slot, Lay::kTmemCols);
    else tc::tmem_alloc(tmem_slot, Lay::kTmemCols);
    tc::fence_before_sync();
  }
  __syncthreads();
  // pairs: the partner's barriers are initialised before copies or commits target them
  if (Src::kPair) tc::cluster_sync();
  tc::fence_after_sync();
  if (threadIdx.x == 0) ISING_TRACE(0);
  const uint32_t tmem_base = *tmem_slot;
  const int total = src.total();

  if (warp == 0 || warp == 2) {
    if (lane == 0) {
      // ------------------------------------------------ TMA producers
      // warp 0 copies the J tiles, warp 2 the S tiles of each stage (one
      // thread issues a TMA copy only every ~250 cycles); each arrives on the
      // stage's full barrier with its own byte count
      const bool jside = warp == 0;
      // J row tiles and spin tiles are read by many CTAs of a step: keep
      // them in L2 ahead of the state, which streams through once
      const uint64_t pol = tc::policy_evict_last();
      uint32_t stage = 0, phase = 0;
      int issued = 0;
      bool ok = true;
      for (int j = 0, tl = src.at(0); tl < total && ok; tl = src.at(++j)) {
        const TileRef T = src.tile(tl);
        if (T.skip) continue;
        const TcArgs& P = src.args(T);
        const int nk = P.nk, nfull = P.nfull, planes = P.planes;
        // k-steps of the ring: k-blocks (fused), else k-blocks of each plane
        const int nkt = fused ? nk : nk * planes;
        const int kps = fused ? 1 : Lay::kKps;
        if (Src::kGlobalMaps) {
          if (jside) {
            for (int p = 0; p < planes; ++p) {
              tc::fence_map_acquire(T.a(p));
              tc::fence_map_acquire(T.j2(p));
            }
          } else {
            tc::fence_map_acquire(T.B);
            tc::fence_map_acquire(T.S2);
          }
        }
        if (issued == 0) tc::prefetch_map(jside ? T.A0 : T.B);
        for (int kt0 = 0; kt0 < nkt; kt0 += kps) {
          if (!tc::mbar_wait(&empty[stage], phase ^ 1, abort_flag, kWaitCycles)) {
            ok = false;
            break;
          }
          uint8_t* sa = smem + stage * kSt;
          const int cnt = nkt - kt0 < kps ? nkt - kt0 : kps;
          // split pairs: every copy of the pair lands on the first CTA's
          // barrier, whose producers expect both CTAs' bytes
          if (!SPLIT || lead)
            tc::mbar_expect_tx(&full[stage], (uint32_t)(fused && jside ? planes : cnt) *
                                                 (jside ? Lay::kA : Lay::kB) * (SPLIT ? 2u : 1u));
          const uint32_t lead_full = SPLIT ? tc::mapa(tc::smem_u32(&full[stage]), 0) : 0u;
          const int plane0 = kt0 / nk, kb0 = kt0 - plane0 * nk;
          if (fused) {
            // k-block kt0 of every plane (slots 0, 1), its spin tile (slot 2)
            const int kb = kt0;
            uint8_t* sb = sa + 2 * Lay::kA;
            if (jside) {
              for (int p = 0; p < planes; ++p) {
                if (SPLIT && !lead)
                  tc::tma_load_2d_to_pair(sa + p * Lay::kA, T.a(p), lead_full, kb * kBK, T.m0, pol);
                else
                  tc::tma_load_2d_hint(sa + p * Lay::kA, T.a(p), &full[stage], kb * kBK, T.m0, pol);
              }
            } else if constexpr (SPLIT) {
              if (lead) tc::tma_load_2d_hint(sb, T.B, &full[stage], kb * kBK, T.n0, pol);
              else tc::tma_load_2d_to_pair(sb, T.B, lead_full, kb * kBK, T.n0 + BN / 2, pol);
            } else if constexpr (Src::kPair) {
              tc::tma_load_2d_mc(sb + src.rank * (BN / 2) * kRowBytes, T.B, &full[stage], kb * kBK,
                                 T.n0 + (int)src.rank * (BN / 2), 0x3, pol);
            } else {
              tc::tma_load_2d_hint(sb, T.B, &full[stage], kb * kBK, T.n0, pol);
            }
          } else if (Lay::kKps == 2 && kb0 + 1 < nfull) {
            // two whole k-blocks of one plane: one copy per operand
            if (jside) tc::tma_load_3d_hint(sa, T.j2(plane0), &full[stage], 0, T.m0, kb0, pol);
            else
              tc::tma_load_3d_hint(sa + Lay::kKps * Lay::kA, T.S2, &full[stage], 0, T.n0, kb0, pol);
          } else {
            for (int u = 0; u < cnt; ++u) {
              const int kt = kt0 + u;
              const int plane = kt / nk, kb = kt - plane * nk;
              if constexpr (SPLIT) {
                // this CTA's J rows and half of the spin tile, kept here (the
                // pair's MMA reads both CTAs' stages where they are)
                if (lead) {
                  if (jside)
                    tc::tma_load_2d_hint(sa, T.a(plane), &full[stage], kb * kBK, T.m0, pol);
                  else
                    tc::tma_load_2d_hint(sa + Lay::kA, T.B, &full[stage], kb * kBK, T.n0, pol);
                } else {
                  if (jside)
                    tc::tma_load_2d_to_pair(sa, T.a(plane), lead_full, kb * kBK, T.m0, pol);
                  else
                    tc::tma_load_2d_to_pair(sa + Lay::kA, T.B, lead_full, kb * kBK,
                                            T.n0 + BN / 2, pol);
                }
              } else if (jside) {
                tc::tma_load_2d_hint(sa + u * Lay::kA, T.a(plane), &full[stage], kb * kBK, T.m0, pol);
              } else if constexpr (Src::kPair) {
                // this CTA's half of the spin tile, to both CTAs of the pair
                tc::tma_load_2d_mc(sa + Lay::kA + src.rank * (BN / 2) * kRowBytes, T.B,
                                   &full[stage], kb * kBK, T.n0 + (int)src.rank * (BN / 2), 0x3, pol);
              } else {
                tc::tma_load_2d_hint(sa + Lay::kKps * Lay::kA + u * Lay::kB, T.B, &full[stage],
                                     kb * kBK, T.n0, pol);
              }
            }
          }
          if (issued == 0 && jside) ISING_TRACE(1);
          ++issued;
          if (++stage == STAGES) { stage = 0; phase ^= 1; }
        }
      }
      if (jside) ISING_TRACE(2);
      if (Src::kPair && ok && jside) {
        // pairs: wait until both CTAs' MMA issuers have released every stage,
        // so that no commit of the partner arrives on this CTA's barriers
        // after it has left (the cluster barrier at the end follows)
        for (int q = 0; q < STAGES && ok; ++q) {
          ok = tc::mbar_wait(&empty[stage], phase ^ 1, abort_flag, kWaitCycles);
          if (++stage == STAGES) { stage = 0; phase ^= 1; }
        }
      }
      if (!ok) {
        // let the copies already issued land before the CTA exits (a phase
        // the other producer never joined gives up after the bounded wait)
        int back = issued < STAGES ? issued : STAGES;
        uint32_t s = stage, ph = phase;
        for (int q = 0; q < back; ++q) {
          if (s == 0) { s = STAGES - 1; ph ^= 1; } else { --s; }
          tc::mbar_wait(&full[s], ph, nullptr, kWaitCycles / 8);
        }
        atomicExch(src.err(), 1);
      }
    }
  } else if (warp == 1 && SPLIT && !lead) {
    // (second CTA of a split pair: the first CTA issues the pair's MMAs)
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------ MMA issuer
      uint32_t stage = 0, phase = 0;
      int it = 0;
      bool ok = true;
      for (int j = 0, tl = src.at(0); tl < total && ok; tl = src.at(++j)) {
        const TileRef T = src.tile(tl);
        if (T.skip) continue;
        const TcArgs& P = src.args(T);
        const int planes = P.planes;
        const int nkt = fused ? P.nk : P.nk * planes;
        const int kps = fused ? 1 : Lay::kKps;
        const uint32_t idesc = op_idesc(BN, FP8, P.f16, SPLIT ? 256 : 128);
        const int buf = it & 1;
        const uint32_t use = (uint32_t)(it >> 1);
        // (split pairs: both CTAs' epilogues release it, from the cluster)
        if (!tc::mbar_wait<SPLIT>(&acc_empty[buf], (use & 1) ^ 1, abort_flag, kWaitCycles)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t d = tmem_base + (uint32_t)(buf * BN);
        for (int kt0 = 0; kt0 < nkt; kt0 += kps) {
          if (!tc::mbar_wait(&full[stage], phase, abort_flag, kWaitCycles)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          if (it == 0 && kt0 == 0) ISING_TRACE(3);
          const uint32_t sb = tc::smem_u32(smem + stage * kSt);
          if (fused) {
            // k-block kt0: plane 0, then plane 1, against the one spin tile
            const uint64_t db = tc::desc_k_sw128(sb + 2 * Lay::kA);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
              if (p >= planes) break;
              const uint64_t da = tc::desc_k_sw128(sb + p * Lay::kA);
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const uint32_t acc = (kt0 > 0 || p > 0 || k > 0) ? 1u : 0u;
                if constexpr (SPLIT) tc::mma_f16_pair(d, da + 2u * k, db + 2u * k, idesc, acc);
                else tc::mma_f16(d, da + 2u * k, db + 2u * k, idesc, acc);
              }
            }
          }
#pragma unroll
          for (int u = 0; u < Lay::kKps; ++u) {
            if (fused) break;
            const int kt = kt0 + u;
            if (kt >= nkt) break;
            // descriptors of the tiles; K step k adds 32 bytes (2 in the >> 4 address field)
            const uint64_t da = tc::desc_k_sw128(sb + u * Lay::kA);
            const uint64_t db = tc::desc_k_sw128(sb + Lay::kKps * Lay::kA + u * Lay::kB);
#pragma unroll
            for (int k = 0; k < 4; ++k) {  // 32 bytes of K per MMA (16 BF16 or 32 E4M3)
              const uint32_t acc = (kt > 0 || k > 0) ? 1u : 0u;
              if constexpr (SPLIT) {
                if (FP8) tc::mma_f8_pair(d, da + 2u * k, db + 2u * k, idesc, acc);
                else tc::mma_f16_pair(d, da + 2u * k, db + 2u * k, idesc, acc);
              } else {
                if (FP8) tc::mma_f8(d, da + 2u * k, db + 2u * k, idesc, acc);
                else tc::mma_f16(d, da + 2u * k, db + 2u * k, idesc, acc);
              }
            }
          }
          // the stage is free once this CTA's MMAs (and, for pairs, the
          // partner's, whose spin half it also holds) have read it; a split
          // pair's MMAs read both CTAs' stages
          if constexpr (SPLIT) tc::mma_commit_pair_mc(&empty[stage], 0x3);
          else if constexpr (Src::kPair) tc::mma_commit_mc(&empty[stage], 0x3);
          else tc::mma_commit(&empty[stage]);
          if (++stage == STAGES) { stage = 0; phase ^= 1; }
        }
        if (ok) {
          if constexpr (SPLIT) tc::mma_commit_pair_mc(&acc_full[buf], 0x3);  // both halves of D
          else tc::mma_commit(&acc_full[buf]);
        }
        ++it;
      }
      ISING_TRACE(4);
      if (!ok) {
        if constexpr (SPLIT) tc::mma_commit_pair(drain);
        else tc::mma_commit(drain);
        tc::mbar_wait(drain, 0, nullptr, kWaitCycles / 8);
        atomicExch(src.err(), 2);
      }
    }
  } else if (warp >= 4) {
    // ------------------------------------------------ epilogue
    const int q = warp & 3;             // TMEM lane quarter of this warp
    const int part = (warp - 4) >> 2;   // which quarter of the tile's columns
    constexpr int kCols = BN / 4;
    if constexpr (MODE == kModeUpdate && Src::kFold) {
      // the previous step's best tracking, a warp per restart over all the
      // launch's epilogue warps, while the MMAs of the first tile run (it
      // reads that step's partial and spin slots, which this step does not
      // write)
      src.template track_prev<FP8 ? kSpinE4M3 : kSpinBF16>(
          (int64_t)blockIdx.x * kEpiWarps + (warp - 4), (int64_t)gridDim.x * kEpiWarps, lane);
    }
    int it = 0;
    for (int j = 0, tl = src.at(0); tl < total; tl = src.at(++j)) {
      const TileRef T = src.tile(tl);
      if (T.skip) continue;
      const TcArgs& P = src.args(T);
      const long long t = P.counters[0] + 1;
      const float2 bc = P.bias[t];
      float* __restrict__ theta = P.theta;
      float* __restrict__ mvec = P.m;
      float* __restrict__ vvec = P.v;
      const uint16_t* __restrict__ Sin = static_cast<const uint16_t*>(T.S);
      uint16_t* __restrict__ Sout = static_cast<uint16_t*>(T.Snext);
      const uint8_t* __restrict__ Sin8 = static_cast<const uint8_t*>(T.S);
      uint8_t* __restrict__ Sout8 = static_cast<uint8_t*>(T.Snext);
      const int my_it = it++;
      const int buf = my_it & 1;
      const uint32_t use = (uint32_t)(my_it >> 1);
      const int mt = T.mt;
      const int64_t m0 = T.m0;
      const int64_t n0 = (int64_t)T.n0 + part * kCols;
      if ((MODE == kModeUpdate || MODE == kModeRelaxed) && P.work && mt == 0 && warp == 4 &&
          lane == 0)
        atomicAdd(P.work, (unsigned long long)min((int64_t)BN, P.B - T.n0));
      if (!tc::mbar_wait(&acc_full[buf], use & 1, abort_flag, kWaitCycles)) {
        atomicExch(src.err(), 3);
        break;
      }
      tc::fence_after_sync();
      if (my_it == 0 && warp == 4 && lane == 0) ISING_TRACE(5);
      const int64_t i = m0 + 32 * q + lane;
      const bool row_ok = i < P.n;
      const float h = row_ok ? P.hf[i] : 0.f;
      const int hi = row_ok ? P.hint[i] : 0;
      const float rs = (P.rowscale && row_ok) ? P.rowscale[i] : 1.f;
      const uint32_t tbase = tmem_base + ((uint32_t)(32 * q) << 16) +
                             (uint32_t)(buf * BN + part * kCols);
#pragma unroll 1
      for (int c0 = 0; c0 < kCols; c0 += kChunk) {
        uint32_t r[kChunk];
        tc::tmem_ld8(tbase + c0, r);
        // state of this chunk's restarts, loaded while the TMEM read lands
        float th[kChunk], mm[kChunk], vv[kChunk], sv[kChunk];
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          const int64_t b = n0 + c0 + j;
          const bool ok = row_ok && b < P.B;
          const int64_t idx = b * P.ld + i;
          th[j] = 0.f;
          mm[j] = 0.f;
          vv[j] = 0.f;
          sv[j] = 0.f;
          if (ok && MODE != kModeCoupling) {
            if (MODE == kModeUpdate || MODE == kModeRelaxed) {
              // the state is read and written once per step: streaming
              // accesses (evict first) leave L2 to the operand tiles. The
              // spins S_t the step consumes are sgn+(sin theta_{t-1}), as
              // every writer of a spin slot makes them (previous update,
              // initial draw, imported state): taken from theta, not loaded
              th[j] = __ldcs(theta + idx);
              mm[j] = __ldcs(mvec + idx);
              vv[j] = __ldcs(vvec + idx);
            } else {
              sv[j] = FP8 ? (Sin8[idx] == 0x38 ? 1.f : -1.f) : ((Sin[idx] & 0x8000u) ? -1.f : 1.f);
            }
          }
        }
        tc::tmem_wait_ld();
        if (c0 + kChunk == kCols) {
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) {
            // split pairs: the first CTA's issuer waits for both epilogues
            if (SPLIT && !lead) tc::mbar_arrive_cluster(tc::mapa(tc::smem_u32(&acc_empty[buf]), 0));
            else tc::mbar_arrive(&acc_empty[buf]);
          }
        }
        float ef[kChunk];
        int eq[kChunk], eh[kChunk];
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          const int64_t b = n0 + c0 + j;
          const bool ok = row_ok && b < P.B;
          const int64_t idx = b * P.ld + i;
          const float G = __uint_as_float(r[j]) * rs;
          ef[j] = 0.f;
          eq[j] = 0;
          eh[j] = 0;
          if (!ok) continue;
          if (MODE == kModeCoupling) {
            P.Gout[idx] = G;
            continue;
          }
          const float sj = (MODE == kModeUpdate || MODE == kModeRelaxed)
                               ? (sin_nonneg(th[j]) ? 1.f : -1.f) : sv[j];
          if (INT_E) {
            eq[j] = (int)sj * __float2int_rn(G);
            eh[j] = (int)sj * hi;
          } else {
            ef[j] = sj * fmaf(P.k.cq, G, P.k.ch * h);
          }
          if (MODE == kModeUpdate || MODE == kModeRelaxed) {
            // (relaxed mode: G = J x_t, and the partials above go unused)
            const float F = fmaf(P.k.cq, G, fmaf(P.k.ch, h, -P.k.mu * sj));
            const float g = cos_proj(th[j]) * F;
            th[j] = adam_update(P.k, bc.x, bc.y, g, th[j], mm[j], vv[j]);
          }
        }
        if (MODE == kModeUpdate || MODE == kModeRelaxed) {
#pragma unroll
          for (int j = 0; j < kChunk; ++j) {
            const int64_t b = n0 + c0 + j;
            if (!row_ok || b >= P.B) continue;
            const int64_t idx = b * P.ld + i;
            __stcs(theta + idx, th[j]);
            __stcs(mvec + idx, mm[j]);
            __stcs(vvec + idx, vv[j]);
            if (FP8) Sout8[idx] = sin_nonneg(th[j]) ? 0x38 : 0xB8;
            else Sout[idx] = pm1_16(sin_nonneg(th[j]), P.f16);
            if (MODE == kModeRelaxed)
              static_cast<uint16_t*>(P.Xnext)[idx] = to_op16(sin_proj(th[j]), P.f16);
          }
        }
        if ((MODE == kModeUpdate || MODE == kModeEnergy) && mt < P.mtiles) {
          // this warp's 32 spins summed per restart; partial row 4 mt + q
          const int64_t b = n0 + c0 + column_of_lane(lane);
          const int64_t o = ((int64_t)mt * 4 + q) * P.B + b;
          if (INT_E) {
            const int tq = column_sums8(eq, lane);
            const int th2 = P.has_h ? column_sums8(eh, lane) : 0;
            if ((lane & 3) == 0 && b < P.B) {
              T.qpart[o] = tq;
              T.hpart[o] = th2;
            }
          } else {
            const float te = column_sums8(ef, lane);
            if ((lane & 3) == 0 && b < P.B) T.epart[o] = te;
          }
        }
      }
    }
  }
  if (warp == 4 && lane == 0) ISING_TRACE(6);
  __syncwarp();
  __syncthreads();
  // pairs: neither CTA leaves while the other may still copy into its shared
  // memory or arrive on its barriers
  if (Src::kPair) tc::cluster_sync();
  if (threadIdx.x == 0) ISING_TRACE(7);
  if constexpr (MODE == kModeUpdate && Src::kFold) src.advance_step();
  if (warp == 1) {
    tc::fence_after_sync();
    if constexpr (SPLIT) tc::tmem_dealloc_pair(tmem_base, Lay::kTmemCols);
    else tc::tmem_dealloc(tmem_base, Lay::kTmemCols);
  }
}
#undef ISING_TRACE

template <int BN, int MODE, bool INT_E, bool FP8>
__global__ void __launch_bounds__(kThreads, 1)
    tc_step_kernel(const __grid_constant__ CUtensorMap tmA0,
                   const __grid_constant__ CUtensorMap tmA1,
                   const __grid_constant__ CUtensorMap tmA2,
                   const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmJ2_0,
                   const __grid_constant__ CUtensorMap tmJ2_1,
                   const __grid_constant__ CUtensorMap tmJ2_2,
                   const __grid_constant__ CUtensorMap tmS2, const __grid_constant__ TcArgs P) {
  const OneInstance<BN> src{P, &tmA0, &tmA1, &tmA2, &tmB, &tmJ2_0, &tmJ2_1, &tmJ2_2, &tmS2};
  step_tiles<BN, MODE, INT_E, FP8>(src);
}

// The same over clusters of two CTAs sharing each spin tile (PairInstance).
template <int BN, int MODE, bool INT_E, bool FP8>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    tc_step_pair_kernel(const __grid_constant__ CUtensorMap tmA0,
                        const __grid_constant__ CUtensorMap tmA1,
                        const __grid_constant__ CUtensorMap tmA2,
                        const __grid_constant__ CUtensorMap tmBh,
                        const __grid_constant__ CUtensorMap tmJ2_0,
                        const __grid_constant__ CUtensorMap tmJ2_1,
                        const __grid_constant__ CUtensorMap tmJ2_2,
                        const __grid_constant__ CUtensorMap tmS2, const __grid_constant__ TcArgs P) {
  const PairInstance<BN> src{P,      &tmA0,   &tmA1,   &tmA2, &tmBh, &tmJ2_0,
                             &tmJ2_1, &tmJ2_2, &tmS2,   &tmBh, tc::cluster_rank()};
  step_tiles<BN, MODE, INT_E, FP8>(src);
}

// The same with the MMAs of each pair issued as one (cta_group::2, M 256).
template <int BN, int MODE, bool INT_E, bool FP8>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    tc_step_split_kernel(const __grid_constant__ CUtensorMap tmA0,
                         const __grid_constant__ CUtensorMap tmA1,
                         const __grid_constant__ CUtensorMap tmA2,
                         const __grid_constant__ CUtensorMap tmBh,
                         const __grid_constant__ CUtensorMap tmJ2_0,
                         const __grid_constant__ CUtensorMap tmJ2_1,
                         const __grid_constant__ CUtensorMap tmJ2_2,
                         const __grid_constant__ CUtensorMap tmS2, const __grid_constant__ TcArgs P) {
  const PairInstance<BN, true> src{P,      &tmA0,   &tmA1, &tmA2, &tmBh, &tmJ2_0,
                                   &tmJ2_1, &tmJ2_2, &tmS2, &tmBh, tc::cluster_rank()};
  step_tiles<BN, MODE, INT_E, FP8>(src);
}

// One step of every member of a pack (the update mode only).
template <int BN, bool INT_E, bool FP8>
__global__ void __launch_bounds__(kThreads, 1)
    tc_pack_kernel(const PackEntry* __restrict__ entries, const int* __restrict__ start, int count,
                   int* err, bool planes2, const TrackArgs* __restrict__ trk,
                   const int64_t* __restrict__ rstart, unsigned long long* done) {
  const PackedInstances<BN> src{entries, start, count, err, planes2, trk, rstart, done};
  step_tiles<BN, kModeUpdate, INT_E, FP8>(src);
}

// 16-bit operand planes of J, [n][ld] each (columns past n are 0):
//   kind 0  one BF16 plane (exact for integer |J| <= 256),
//   kind 1  FP16 planes of J_ij * 2^e_i: hi = fp16(x), lo = fp16(x - hi) when
//           planes == 2; with the power-of-two row exponents e_i of
//           `rowscale` (2^-e_i per row, from row_pow2_scale_kernel) or e_i = 0
//           when it is null. Each rounding is to nearest, so
//           |x - hi - lo| <= 2^-22 |x| + 2^-25 (the smallest FP16 subnormal is 2^-24).
__global__ void to_planes_kernel(const void* J, int dt, int64_t n, int64_t ld, int kind, int planes,
                                 const float* rowscale, uint16_t* p0, uint16_t* p1) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * ld;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ld, k = e - i * ld;
    double x = k < n ? load_as_double(J, dt, i * n + k) : 0.0;
    if (kind == 0) {
      p0[e] = __bfloat16_as_ushort(__double2bfloat16(x));
      continue;
    }
    if (rowscale) x = x / (double)rowscale[i];  // exact: a power of two
    const __half hi = __double2half(x);
    p0[e] = __half_as_ushort(hi);
    if (planes == 2) p1[e] = __half_as_ushort(__double2half(x - (double)__half2float(hi)));
  }
}

// Per-row power-of-two scales for the FP16 planes: with a_i = max_j |J_ij|,
// scale_i = 2^(E_i - 15) where a_i = f 2^E_i, f in [0.5, 1), so that
// a_i / scale_i lies in [2^14, 2^15) (below the FP16 maximum 65504, and the
// low plane stays clear of the subnormal range); 1 for an all-zero row. The
// epilogue multiplies the accumulated product of row i by scale_i, exactly.
__global__ void row_pow2_scale_kernel(const void* J, int dt, int64_t n, float* scale) {
  __shared__ double sm[32];
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    double mx = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) mx = fmax(mx, fabs(load_as_double(J, dt, i * n + k)));
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, sm[w]);
      mx = fmax(mx, sm[0]);
      int ex = 15;
      if (mx > 0.0) frexp(mx, &ex);
      scale[i] = ldexpf(1.0f, min(max(ex - 15, -126), 127));
    }
    __syncthreads();
  }
}

// E4M3 plane: exact when rowscale is null (integers |J| <= 16), otherwise
// J_ij / scale_i rounded to E4M3 with scale_i = max_j |J_ij| / 448.
__global__ void to_fp8_kernel(const void* J, int dt, int64_t n, int64_t ld, const float* rowscale,
                              uint8_t* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * ld;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ld, k = e - i * ld;
    double x = k < n ? load_as_double(J, dt, i * n + k) : 0.0;
    if (rowscale) x = rowscale[i] > 0.f ? x / (double)rowscale[i] : 0.0;
    out[e] = (uint8_t)__nv_cvt_float_to_fp8((float)x, __NV_SATFINITE, __NV_E4M3);
  }
}

// max_i sum_j |J_ij| of an integer-valued dense J (exact in FP64), one warp per row.
__global__ void row_abssum_max_kernel(const void* J, int dt, int64_t n, unsigned long long* out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    double a = 0.0;
    for (int64_t k = lane; k < n; k += 32) a += fabs(load_as_double(J, dt, i * n + k));
    for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) atomicMax(out, (unsigned long long)a);
  }
}

__global__ void row_absmax_kernel(const void* J, int dt, int64_t n, float* scale) {
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    double mx = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) mx = fmax(mx, fabs(load_as_double(J, dt, i * n + k)));
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ double sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, sm[w]);
      scale[i] = (float)(sm[0] > mx ? sm[0] : mx) / 448.f;
    }
    __syncthreads();
  }
}


// ---------------------------------------------------------------------------
// Resident form: when every tile of the problem fits one CTA per SM, each CTA
// keeps its tile of theta, m, v in tensor memory for a whole run of steps, so
// a step moves only the J / S tiles (TMA) and the new spins and energy
// partials (global stores). A CTA holds two groups of GN restarts, each with
// its own tensor-memory block (accumulator, theta, m, v: columns
// [4 GN g, 4 GN (g + 1))), and the tensor cores alternate between them: while
// the epilogue warps update group 0 from its accumulator, the MMAs of group 1
// run, and the other way round, so the MMA stream (paced by one thread's issue
// rate) and the epilogue (bound by instruction issue) overlap. Step t + 1 of
// a group needs S_t of all rows, i.e. the output of every m-tile of the same
// restarts, so the CTAs of one group's column pass a barrier between steps
// (an arrival counter per group and column; the cooperative launch keeps all
// CTAs co-resident, and the waits are bounded); groups and columns run
// independently. After a group's barrier its controller warp tracks the best
// of that step for the CTA's slice of the group's restarts. The spins a step
// consumes are the signs of theta the epilogue kept in a register since the
// previous update (derived from theta when the launch starts), so the
// epilogue reads no state from global memory.

struct TcResArgs {
  TcArgs P;
  int64_t steps;
  void* spins[3];
  long long* qpart[2];
  long long* hpart[2];
  float* epart[2];
  unsigned int* gbar;  // per restart-column barrier arrivals, 32 words apart (zeroed before the launch)
  int* gabort;         // raised by any CTA that gives up
  double* best_E;
  long long* best_t;
  int8_t* best_s;
  double* last_E;
  int64_t bs_ld;       // row pitch of best_s
  double cq, chs;      // E = cq * Q + chs * H (integer mode)
  int rows;            // energy-partial rows (4 per m-tile)
  int64_t T;           // steps of the run (convergence rule: steps <= T feed it)
  double* conv_ring;   // convergence rule state, or null (see conv_update)
  double* conv_init;
  long long* conv_step;
  unsigned long long* conv_count;
  int jres;            // J tiles (k-blocks) kept in shared memory for the whole run
  int nst;             // pipeline stages after them
  uint32_t bars;       // shared-memory offset of the barrier block
  int slice;           // restarts of a group tracked per CTA of its column
  int nfull;           // k-blocks lying wholly below column n (pairs of them load as one box)
};

// Best tracking of step t for restarts [b0, b1) by one warp, a lane per
// restart, with the same sums as track_kernel (whose lane l adds rows l,
// l + 32, ... starting from 0, then combines the lanes by an xor tree over
// lane bits 4, 3, 2, 1, 0): here one lane forms the 32 lane sums and adds
// them in that tree's order. The spins of the improved restarts are then
// copied one restart at a time by the whole warp. With the convergence rule a
// stopped restart is left alone, and steps t <= T feed the rule.
template <bool INT_E, bool FP8>
__device__ __forceinline__ void track_warp(const TcResArgs& R, long long t, int64_t b0, int64_t b1,
                                           int lane) {
  const TcArgs& P = R.P;
  const int ps = (int)(t % 2);
  const void* St = R.spins[t % 3];
  for (int64_t bb = b0; bb < b1; bb += 32) {
    const int64_t b = bb + lane;
    const bool ok = b < b1;
    bool improved = false;
    const bool active = ok && (R.conv_step == nullptr || R.conv_step[b] == 0);
    if (active) {
      const double best = R.best_E[b];
      double E;
      if (INT_E) {
        long long q = 0, hs = 0;
        for (int r = 0; r < R.rows; ++r) {
          q += R.qpart[ps][(int64_t)r * P.B + b];
          hs += R.hpart[ps][(int64_t)r * P.B + b];
        }
        E = R.cq * (double)q + R.chs * (double)hs;
      } else {
        double y[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          double lo = 0.0, hi = 0.0;  // the sums of lanes j and j + 16
          for (int r = j; r < R.rows; r += 32) lo += (double)R.epart[ps][(int64_t)r * P.B + b];
          for (int r = j + 16; r < R.rows; r += 32) hi += (double)R.epart[ps][(int64_t)r * P.B + b];
          y[j] = lo + hi;
        }
#pragma unroll
        for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
          for (int j = 0; j < w; ++j) y[j] = y[j] + y[j + w];
        E = y[0];
      }
      improved = E < best;
      R.last_E[b] = E;
      if (improved) {
        R.best_E[b] = E;
        R.best_t[b] = t;
      }
      if (R.conv_step && t <= R.T)
        conv_update(R.conv_ring, R.conv_init, R.conv_step, R.conv_count, P.B, b, t, E);
    }
    for (unsigned int m = __ballot_sync(0xffffffffu, improved); m; m &= m - 1) {
      const int64_t br = bb + __ffs(m) - 1;
      copy_spin_row_dense<FP8 ? kSpinE4M3 : kSpinBF16>(R.best_s + br * R.bs_ld, St, P.n, P.ld, br, lane);
    }
  }
}

// Per-lane constants of the resident epilogue: the lane owns row i of the
// tile and the warp's BN / 4 columns starting at restart nb0.
struct EpiLane {
  int64_t i, orow;
  bool row_ok;
  int hi, lane;
  float rs, chh, hm_pos, hm_neg;
};

// The warp's columns within one restart group: first restart, how many of
// them lie below B, tensor-memory column of their accumulator.
struct EpiGroup {
  int64_t nb0;
  int ncols;
  uint32_t t_acc;
};

// One step of the resident epilogue over the warp's columns, in chunks of 8:
// the step's energy partials, the Adam update of theta / m / v (kept in
// tensor memory), and the next spins. Rows past n and columns past B hold
// G = 0 (the TMA fills out-of-range operand rows with zeros), so their
// energy terms vanish or are never stored; only stores are guarded.
// EMODE 1 (integer G with |G| < 2^22): s_i G_i is turned into an integer by
// adding 1.5 * 2^23 in FP32, whose bit pattern is then 0x4B400000 + s_i G_i,
// so the warp sums the raw patterns (redux.sync, wrapping) and removes 32
// times the offset once per column. EMODE 2 (also 32 max_i sum_j |J_ij| <
// 2^15): two columns share one reduction, packed as a + 2^16 b; the low half
// of the sum is then sum a exactly and the high half sum b. EMODE 0 converts
// with F2I. `sbits` holds the signs of this lane's theta (bit sh + c: column
// c of the warp's columns in this group): the spins the step consumes, kept
// from the previous step instead of evaluated again, and replaced by the new
// ones.
template <int GN, bool INT_E, bool FP8, int EMODE>
__device__ __forceinline__ void resident_chunks(const TcResArgs& R, const EpiLane& E,
                                                const EpiGroup& Gr, long long t, float2 bc,
                                                bool last, uint64_t* acc_empty, uint32_t& sbits,
                                                int sh) {
  const TcArgs& P = R.P;
  constexpr int kCols = GN / 4;
  const uint32_t t_th = Gr.t_acc + GN, t_m = Gr.t_acc + 2 * GN, t_v = Gr.t_acc + 3 * GN;
  void* Sout = R.spins[(t + 1) % 3];
  const int ps = (int)(t % 2);
  const int lane = E.lane;
#pragma unroll 1
  for (int c0 = 0; c0 < kCols; c0 += kChunk) {
    uint32_t r[kChunk], th[kChunk], mm[kChunk], vv[kChunk];
    tc::tmem_ld8(Gr.t_acc + c0, r);
    tc::tmem_ld8(t_th + c0, th);
    tc::tmem_ld8(t_m + c0, mm);
    tc::tmem_ld8(t_v + c0, vv);
    tc::tmem_wait_ld();
    if (c0 + kChunk == kCols) {
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(acc_empty);
    }
    const uint32_t pos_bits = (sbits >> (sh + c0)) & 0xFFu;  // the spins this step consumes
    uint32_t new_bits = 0;
    int eq[kChunk];
    float ef[kChunk];
#pragma unroll
    for (int j = 0; j < kChunk; ++j) {
      float tj = __uint_as_float(th[j]), mj = __uint_as_float(mm[j]), vj = __uint_as_float(vv[j]);
      const float G = INT_E ? __uint_as_float(r[j]) : __uint_as_float(r[j]) * E.rs;
      const bool pos = (pos_bits >> j) & 1u;
      if (INT_E) {
        if (EMODE > 0) {
          eq[j] = __float_as_int(__fadd_rn(pos ? G : -G, 12582912.0f));
        } else {
          const int gi = __float2int_rn(G);
          eq[j] = pos ? gi : -gi;
        }
      } else {
        ef[j] = (pos ? 1.f : -1.f) * fmaf(P.k.cq, G, E.chh);
      }
      const float F = fmaf(P.k.cq, G, pos ? E.hm_pos : E.hm_neg);
      const float g = cos_proj(tj) * F;
      tj = adam_update(P.k, bc.x, bc.y, g, tj, mj, vj);
      new_bits |= (sin_nonneg(tj) ? 1u : 0u) << j;
      th[j] = __float_as_uint(tj);
      mm[j] = __float_as_uint(mj);
      vv[j] = __float_as_uint(vj);
    }
    sbits = (sbits & ~(0xFFu << (sh + c0))) | (new_bits << (sh + c0));
    if (!last) {
      tc::tmem_st8(t_th + c0, th);
      tc::tmem_st8(t_m + c0, mm);
      tc::tmem_st8(t_v + c0, vv);
    }
    if (E.row_ok) {
      const int nv = Gr.ncols - c0;  // columns of this chunk below B
      const int64_t base = (Gr.nb0 + c0) * P.ld + E.i;
      if (nv >= kChunk) {
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          const bool sp = (new_bits >> j) & 1u;
          if (FP8) static_cast<uint8_t*>(Sout)[base + j * P.ld] = sp ? 0x38 : 0xB8;
          else static_cast<uint16_t*>(Sout)[base + j * P.ld] = pm1_16(sp, P.f16);
        }
      } else {
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          if (j >= nv) break;
          const bool sp = (new_bits >> j) & 1u;
          if (FP8) static_cast<uint8_t*>(Sout)[base + j * P.ld] = sp ? 0x38 : 0xB8;
          else static_cast<uint16_t*>(Sout)[base + j * P.ld] = pm1_16(sp, P.f16);
        }
      }
      if (last) {
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          if (j >= nv) break;
          const int64_t idx = base + (int64_t)j * P.ld;
          P.theta[idx] = __uint_as_float(th[j]);
          P.m[idx] = __uint_as_float(mm[j]);
          P.v[idx] = __uint_as_float(vv[j]);
        }
      }
    }
    if (INT_E) {
      // lane j < 8 ends up with the sums of column c0 + j over the warp's 32 rows
      int q = 0, hs = 0;
      if (EMODE == 2) {
#pragma unroll
        for (int jp = 0; jp < kChunk / 2; ++jp) {
          // 0x4B400000 << 16 wraps to 0: only the low column carries the offset
          const unsigned int v = (unsigned int)eq[2 * jp] + ((unsigned int)eq[2 * jp + 1] << 16);
          const unsigned int sum = __reduce_add_sync(0xffffffffu, v) - 32u * 0x4B400000u;
          const int lo = (int)(short)(sum & 0xFFFFu);
          const int hi = (int)(sum - (unsigned int)lo) >> 16;
          if (lane == 2 * jp) q = lo;
          if (lane == 2 * jp + 1) q = hi;
        }
      } else {
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          const unsigned int sum = __reduce_add_sync(0xffffffffu, (unsigned int)eq[j]);
          if (lane == j) q = (int)(EMODE == 1 ? sum - 32u * 0x4B400000u : sum);
        }
      }
      if (P.has_h) {
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          const int hv = ((pos_bits >> j) & 1u) ? E.hi : -E.hi;
          const int sum = __reduce_add_sync(0xffffffffu, hv);
          if (lane == j) hs = sum;
        }
      }
      const int64_t b = Gr.nb0 + c0 + lane;
      if (lane < kChunk && b < P.B) {
        R.qpart[ps][E.orow + b] = q;
        R.hpart[ps][E.orow + b] = hs;
      }
    } else {
      const float te = column_sums8(ef, lane);
      const int64_t b = Gr.nb0 + c0 + column_of_lane(lane);
      if ((lane & 3) == 0 && b < P.B) R.epart[ps][E.orow + b] = te;
    }
  }
}

template <int GN, bool INT_E, bool FP8>
__global__ void __launch_bounds__(kThreads, 1)
    tc_resident_kernel(const __grid_constant__ CUtensorMap tmA0,
                       const __grid_constant__ CUtensorMap tmA1,
                       const __grid_constant__ CUtensorMap tmA2,
                       const __grid_constant__ CUtensorMap tmB0,
                       const __grid_constant__ CUtensorMap tmB1,
                       const __grid_constant__ CUtensorMap tmB2,
                       const __grid_constant__ CUtensorMap tmJ2_0,
                       const __grid_constant__ CUtensorMap tmJ2_1,
                       const __grid_constant__ CUtensorMap tmJ2_2,
                       const __grid_constant__ CUtensorMap tmS2_0,
                       const __grid_constant__ CUtensorMap tmS2_1,
                       const __grid_constant__ CUtensorMap tmS2_2, const TcResArgs R) {
  const TcArgs& P = R.P;
  using Lay = ResLayout<GN>;
  const int STAGES = R.nst;
  const int jres = R.jres;
  constexpr int kBK = FP8 ? 128 : 64;
  constexpr uint32_t kTmemCols = 8 * GN;  // per group: accumulator, theta, m, v
  constexpr int kCols = GN / 4;           // columns of a group per epilogue warp
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* stages = smem + (size_t)jres * Lay::kA;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + R.bars);
  uint64_t* empty = full + Lay::kMaxStages;
  uint64_t* jfull = empty + Lay::kMaxStages;  // the resident J tiles have landed
  uint64_t* acc_full = jfull + 1;       // [2], one per restart group
  uint64_t* acc_empty = acc_full + 2;   // [2]
  uint64_t* step_done = acc_empty + 2;  // [2]
  uint64_t* go = step_done + 2;         // [2]
  uint64_t* drain = go + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int g = 0; g < 2; ++g) {
      tc::mbar_init(&acc_full[g], 1);
      tc::mbar_init(&acc_empty[g], kEpiWarps);
      tc::mbar_init(&step_done[g], kEpiWarps);
      tc::mbar_init(&go[g], 1);
    }
    tc::mbar_init(drain, 1);
    tc::mbar_init(jfull, 1);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, kTmemCols);
    tc::fence_before_sync();
  }
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem_base = *tmem_slot;
  const long long t0 = P.counters[0];
  const int64_t K = R.steps;
  const int64_t NP = 2 * K;  // phases: step s of group g is phase 2 s + g
  const int mt = blockIdx.x % P.mtiles;
  const int64_t m0 = (int64_t)mt * kBM;
  const int64_t n0 = (int64_t)(blockIdx.x / P.mtiles) * (2 * GN);  // first restart of the CTA
  const int nkt = P.nk * P.planes;
  // role timeline of one step of group 0 (profiling): 0 producer starts the
  // step, 1 last TMA issued, 2 last MMA committed, 3 controller finished
  // tracking the step, 4 epilogue has the accumulator, 5 epilogue done,
  // 6 controller saw the CTA done, 7 column barrier passed
  const int64_t rec = K >= 2 ? K - 2 : 0;
#define ISING_RTRACE(slot, s, g)                                                   \
  do {                                                                             \
    if (P.trace && (s) == rec && (g) == 0)                                         \
      P.trace[(size_t)blockIdx.x * 8 + (slot)] = now_ns();                          \
  } while (0)

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------ TMA producer
      // the resident J tiles, once
      if (jres > 0) {
        tc::mbar_expect_tx(jfull, (uint32_t)jres * Lay::kA);
        // (unit kt of a step is plane kt % planes of k-block kt / planes: the
        // planes k-block by k-block, the order of every form)
        for (int kt = 0; kt < jres; ++kt) {
          const int plane = kt % P.planes, kb = kt / P.planes;
          const CUtensorMap* ma = plane == 0 ? &tmA0 : (plane == 1 ? &tmA1 : &tmA2);
          tc::tma_load_2d(smem + (size_t)kt * Lay::kA, ma, jfull, kb * kBK, (int)m0);
        }
      }
      uint32_t stage = 0, phase = 0;
      int issued = 0;
      bool ok = true;
      for (int64_t p = 0; p < NP && ok; ++p) {
        const int64_t s = p >> 1;
        const int g = (int)(p & 1);
        const long long t = t0 + s + 1;
        const int slot = (int)(t % 3);
        const CUtensorMap* mb = slot == 0 ? &tmB0 : (slot == 1 ? &tmB1 : &tmB2);
        const CUtensorMap* mb2 = slot == 0 ? &tmS2_0 : (slot == 1 ? &tmS2_1 : &tmS2_2);
        const int nb = (int)(n0 + g * GN);
        if (s > 0) {
          // S_t of the group exists once every CTA of its column is through step t - 1
          if (!tc::mbar_wait(&go[g], (uint32_t)((s - 1) & 1), abort_flag, kWaitCycles)) {
            ok = false;
            break;
          }
          tc::fence_proxy_async_global();
        }
        ISING_RTRACE(0, s, g);
        for (int kt0 = 0; kt0 < nkt; kt0 += Lay::kKps) {
          if (!tc::mbar_wait(&empty[stage], phase ^ 1, abort_flag, kWaitCycles)) {
            ok = false;
            break;
          }
          uint8_t* sa = stages + (size_t)stage * Lay::kStage;
          uint32_t bytes = 0;
#pragma unroll
          for (int u = 0; u < Lay::kKps; ++u) {
            const int kt = kt0 + u;
            if (kt < nkt) bytes += kt < jres ? Lay::kB : Lay::kA + Lay::kB;
          }
          tc::mbar_expect_tx(&full[stage], bytes);
          const int plane0 = kt0 % P.planes, kb0 = kt0 / P.planes;
          if (P.planes == 1 && kb0 + 1 < R.nfull) {
            // two whole k-blocks of one plane: one box each for J and S (the
            // issue of a TMA instruction, not its bytes, paces this thread)
            if (kt0 >= jres) {
              const CUtensorMap* ma = plane0 == 0 ? &tmJ2_0 : (plane0 == 1 ? &tmJ2_1 : &tmJ2_2);
              tc::tma_load_3d(sa, ma, &full[stage], 0, (int)m0, kb0);
            } else if (kt0 + 1 >= jres) {
              const CUtensorMap* ma = plane0 == 0 ? &tmA0 : (plane0 == 1 ? &tmA1 : &tmA2);
              tc::tma_load_2d(sa + Lay::kA, ma, &full[stage], (kb0 + 1) * kBK, (int)m0);
            }
            tc::tma_load_3d(sa + Lay::kKps * Lay::kA, mb2, &full[stage], 0, nb, kb0);
          } else {
#pragma unroll
            for (int u = 0; u < Lay::kKps; ++u) {
              const int kt = kt0 + u;
              if (kt >= nkt) break;
              const int plane = kt % P.planes, kb = kt / P.planes;
              if (kt >= jres) {
                const CUtensorMap* ma = plane == 0 ? &tmA0 : (plane == 1 ? &tmA1 : &tmA2);
                tc::tma_load_2d(sa + u * Lay::kA, ma, &full[stage], kb * kBK, (int)m0);
              }
              tc::tma_load_2d(sa + Lay::kKps * Lay::kA + u * Lay::kB, mb, &full[stage], kb * kBK, nb);
            }
          }
          ++issued;
          if (++stage == (uint32_t)STAGES) { stage = 0; phase ^= 1; }
        }
        ISING_RTRACE(1, s, g);
      }
      if (!ok) {
        int back = issued < STAGES ? issued : STAGES;
        uint32_t s2 = stage, ph = phase;
        for (int q = 0; q < back; ++q) {
          if (s2 == 0) { s2 = STAGES - 1; ph ^= 1; } else { --s2; }
          tc::mbar_wait(&full[s2], ph, nullptr, kWaitCycles / 8);
        }
        if (jres > 0) tc::mbar_wait(jfull, 0, nullptr, kWaitCycles / 8);
        atomicExch(P.err, 1);
        atomicExch(R.gabort, 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------ MMA issuer
      const uint32_t idesc = op_idesc(GN, FP8, P.f16);
      uint32_t stage = 0, phase = 0;
      bool ok = jres == 0 || tc::mbar_wait(jfull, 0, abort_flag, kWaitCycles);
      for (int64_t p = 0; p < NP && ok; ++p) {
        const int64_t s = p >> 1;
        const int g = (int)(p & 1);
        const uint32_t d = tmem_base + (uint32_t)(g * 4 * GN);
        if (!tc::mbar_wait(&acc_empty[g], (uint32_t)((s & 1) ^ 1), abort_flag, kWaitCycles)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        for (int kt0 = 0; kt0 < nkt; kt0 += Lay::kKps) {
          if (!tc::mbar_wait(&full[stage], phase, abort_flag, kWaitCycles)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sb = tc::smem_u32(stages + (size_t)stage * Lay::kStage);
#pragma unroll
          for (int u = 0; u < Lay::kKps; ++u) {
            const int kt = kt0 + u;
            if (kt >= nkt) break;
            const uint32_t a0 = kt < jres ? tc::smem_u32(smem + (size_t)kt * Lay::kA) : sb + u * Lay::kA;
            // descriptors of the tiles; K step k adds 32 bytes (2 in the >> 4 address field)
            const uint64_t da = tc::desc_k_sw128(a0);
            const uint64_t db = tc::desc_k_sw128(sb + Lay::kKps * Lay::kA + u * Lay::kB);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              if (FP8)
                tc::mma_f8(d, da + 2u * k, db + 2u * k, idesc,
                           (kt > 0 || k > 0) ? 1u : 0u);
              else
                tc::mma_f16(d, da + 2u * k, db + 2u * k, idesc,
                            (kt > 0 || k > 0) ? 1u : 0u);
            }
          }
          tc::mma_commit(&empty[stage]);
          if (++stage == (uint32_t)STAGES) { stage = 0; phase ^= 1; }
        }
        if (ok) tc::mma_commit(&acc_full[g]);
        ISING_RTRACE(2, s, g);
      }
      if (!ok) {
        tc::mma_commit(drain);
        tc::mbar_wait(drain, 0, nullptr, kWaitCycles / 8);
        atomicExch(P.err, 2);
        atomicExch(R.gabort, 1);
      }
    }
  } else if (warp == 2 || warp == 3) {
    // ------------------------------------------------ column-barrier controller
    // of group g = warp - 2, and its best tracking: the CTAs of one restart
    // group's column (all m-tiles of the same restarts) exchange spins;
    // groups and columns are independent and never wait on each other. Step
    // s of the group is tracked after its barrier, before this CTA arrives at
    // the barrier of step s + 1, which any overwrite of the step's partials
    // and spins (at step s + 2) has to wait for.
    const int g = warp - 2;
    unsigned int* colbar = R.gbar + 32 * (2 * (blockIdx.x / P.mtiles) + g);
    const int64_t gs = n0 + g * GN;
    const int64_t ge = gs + GN < P.B ? gs + GN : P.B;
    const int64_t tb0 = gs + (int64_t)mt * R.slice;
    const int64_t tb1 = tb0 + R.slice < ge ? tb0 + R.slice : ge;
    for (int64_t s = 0; s < K; ++s) {
      int ok = 1;
      if (lane == 0) ok = tc::mbar_wait(&step_done[g], (uint32_t)(s & 1), abort_flag, kWaitCycles) ? 1 : 0;
      if (lane == 0 && ok) {
        ISING_RTRACE(6, s, g);
        // release at GPU scope: the spins and partials this CTA's epilogue
        // wrote (ordered before step_done) are visible before the arrival
        tc::red_release_gpu(colbar, 1u);
        const unsigned int target = (unsigned int)(s + 1) * (unsigned int)P.mtiles;
        const long long c0 = clock64();
        while (tc::ld_acquire_gpu(colbar) < target) {
          if (*reinterpret_cast<volatile int*>(R.gabort)) { ok = 0; break; }
          if (clock64() - c0 > kWaitCycles) {
            atomicExch(R.gabort, 1);
            atomicExch(P.err, 4);
            ok = 0;
            break;
          }
        }
        if (!ok) *abort_flag = 1;
        else {
          ISING_RTRACE(7, s, g);
          tc::mbar_arrive(&go[g]);
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      // acquire side of the barrier for the whole warp (lane 0's acquire
      // load is ordered before the shuffle)
      __threadfence();
      track_warp<INT_E, FP8>(R, t0 + s + 1, tb0, tb1, lane);
      if (lane == 0) ISING_RTRACE(3, s, g);
    }
  } else {
    // ------------------------------------------------ epilogue
    const int q = warp & 3;
    const int part = (warp - 4) >> 2;  // which quarter of a group's columns
    const int64_t i = m0 + 32 * q + lane;
    const bool row_ok = i < P.n;
    const float h = row_ok ? P.hf[i] : 0.f;
    EpiLane E;
    E.i = i;
    E.row_ok = row_ok;
    E.hi = row_ok ? P.hint[i] : 0;
    E.rs = (P.rowscale && row_ok) ? P.rowscale[i] : 1.f;
    E.chh = P.k.ch * h;
    E.hm_pos = fmaf(P.k.ch, h, -P.k.mu);  // = fmaf(ch, h, -mu s) for s = +1
    E.hm_neg = fmaf(P.k.ch, h, P.k.mu);   // ... and for s = -1
    E.orow = ((int64_t)mt * 4 + q) * P.B;
    E.lane = lane;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    auto group = [&](int g) {
      EpiGroup Gr;
      Gr.nb0 = n0 + g * GN + part * kCols;
      Gr.ncols = (int)max((int64_t)0, min((int64_t)kCols, P.B - Gr.nb0));
      Gr.t_acc = tmem_base + lane_off + (uint32_t)(g * 4 * GN + part * kCols);
      return Gr;
    };
    // state of this warp's columns into tensor memory, and the signs of theta
    // (bit g kCols + c for column c of group g)
    uint32_t sbits = 0;
    for (int g = 0; g < 2; ++g) {
      const EpiGroup Gr = group(g);
#pragma unroll 1
      for (int c0 = 0; c0 < kCols; c0 += kChunk) {
        uint32_t a[kChunk], bm[kChunk], c[kChunk];
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          const int64_t b = Gr.nb0 + c0 + j;
          const bool ok = row_ok && b < P.B;
          const int64_t idx = b * P.ld + i;
          const float th0 = ok ? P.theta[idx] : 0.f;
          a[j] = __float_as_uint(th0);
          bm[j] = __float_as_uint(ok ? P.m[idx] : 0.f);
          c[j] = __float_as_uint(ok ? P.v[idx] : 0.f);
          sbits |= (sin_nonneg(th0) ? 1u : 0u) << (g * kCols + c0 + j);
        }
        tc::tmem_st8(Gr.t_acc + GN + c0, a);
        tc::tmem_st8(Gr.t_acc + 2 * GN + c0, bm);
        tc::tmem_st8(Gr.t_acc + 3 * GN + c0, c);
      }
    }
    tc::tmem_wait_st();
    bool ok = true;
    for (int64_t p = 0; p < NP && ok; ++p) {
      const int64_t s = p >> 1;
      const int g = (int)(p & 1);
      const long long t = t0 + s + 1;
      const float2 bc = P.bias[t];  // loaded ahead of the wait, off the critical path
      if (!tc::mbar_wait(&acc_full[g], (uint32_t)(s & 1), abort_flag, kWaitCycles)) {
        atomicExch(P.err, 3);
        atomicExch(R.gabort, 1);
        ok = false;
        break;
      }
      tc::fence_after_sync();
      if (warp == 4 && lane == 0) ISING_RTRACE(4, s, g);
      const bool last = s + 1 == K;
      const EpiGroup Gr = group(g);
      if constexpr (INT_E) {
        if (P.gmagic == 2)
          resident_chunks<GN, true, FP8, 2>(R, E, Gr, t, bc, last, &acc_empty[g], sbits, g * kCols);
        else if (P.gmagic == 1)
          resident_chunks<GN, true, FP8, 1>(R, E, Gr, t, bc, last, &acc_empty[g], sbits, g * kCols);
        else
          resident_chunks<GN, true, FP8, 0>(R, E, Gr, t, bc, last, &acc_empty[g], sbits, g * kCols);
      } else {
        resident_chunks<GN, false, FP8, 0>(R, E, Gr, t, bc, last, &acc_empty[g], sbits, g * kCols);
      }
      tc::tmem_wait_st();
      tc::fence_proxy_async_global();
      __syncwarp();
      if (warp == 4 && lane == 0) ISING_RTRACE(5, s, g);
      if (lane == 0) tc::mbar_arrive(&step_done[g]);
    }
  }
#undef ISING_RTRACE
  __syncwarp();
  __syncthreads();
  if (threadIdx.x == 0 && blockIdx.x == 0 && !*abort_flag) {
    long long* cnt = const_cast<long long*>(P.counters);
    cnt[0] = t0 + K;
  }
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem_base, kTmemCols);
  }
}


// ---------------------------------------------------------------------------
// Small form: when all n <= 128 spins fit one row tile, every CTA holds all of
// J in shared memory (loaded once) for its block of BN restarts, so a step
// needs nothing from other CTAs. The epilogue writes the next spins straight
// into the shared-memory B operand, in the 128-byte swizzled layout the TMA
// produces (16-byte chunk c of row r stored at chunk c ^ (r mod 8)); after a
// proxy fence and the step's one CTA barrier the tensor cores read them. No
// grid barrier and no global round trip per step: warp 0 issues TMA and MMAs
// and, while the tensor cores run step s, turns the energy partials of step
// s - 1 into energies and bests; warps 1..16 run the epilogue (TMEM lane
// quarter warp mod 4) and keep, per column, the spins of the best step as bits
// in a register (updated two steps late, when the improvement bits are known),
// written to global memory once at the end of the launch.

constexpr int kSmallEpi = 16;
constexpr int kSmallThreads = 32 * (1 + kSmallEpi);

struct TcSmallArgs {
  TcArgs P;
  int64_t steps;
  long long t0;       // steps already taken (the first step here is t0 + 1)
  void* spins_out;    // global slot receiving S_{t0+K+1}, [B][ld]
  double* best_E;
  long long* best_t;
  int8_t* best_s;
  double* last_E;
  int64_t bs_ld;
  double cq, chs;     // E = cq * Q + chs * H (integer mode)
};

// Byte offset of element (row r, K index k) in a swizzled operand tile whose
// rows hold kBK elements of `esize` bytes (128 bytes).
__device__ __forceinline__ uint32_t swz_offset(int r, int k, int esize) {
  const uint32_t byte = (uint32_t)k * (uint32_t)esize;
  return (uint32_t)r * 128u + ((((byte >> 4) ^ (uint32_t)(r & 7)) << 4) | (byte & 15u));
}

template <int BN, bool FP8>
struct SmallLayout {
  static constexpr int kBK = FP8 ? 128 : 64;
  static constexpr uint32_t kA = kBM * kRowBytes;  // one J k-block tile
  static constexpr uint32_t kSk = BN * kRowBytes;  // one S k-block tile
};

template <int BN, bool INT_E, bool FP8>
__global__ void __launch_bounds__(kSmallThreads, 1)
    tc_small_kernel(const __grid_constant__ CUtensorMap tmA0,
                    const __grid_constant__ CUtensorMap tmA1,
                    const __grid_constant__ CUtensorMap tmA2,
                    const __grid_constant__ CUtensorMap tmB, const TcSmallArgs R) {
  using Lay = SmallLayout<BN, FP8>;
  constexpr int kBK = Lay::kBK;
  constexpr int esize = FP8 ? 1 : 2;
  constexpr uint32_t kTmemCols = 4 * BN;
  constexpr int kCols = BN / 4;  // columns of one epilogue warp (8, 16 or 32)
  constexpr int kWords = BN / 32;
  const TcArgs& P = R.P;
  const int nk = P.nk, nkt = P.nk * P.planes;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* Jsm = smem;                                    // nkt x kA
  uint8_t* Ssm = Jsm + (size_t)nkt * Lay::kA;             // 2 buffers x nk x kSk
  const size_t kSbuf = (size_t)nk * Lay::kSk;
  int* part_q = reinterpret_cast<int*>(Ssm + 2 * kSbuf);  // [2][4][BN] (slot s mod 2)
  int* part_h = part_q + 8 * BN;                          // [2][4][BN]
  float* part_f = reinterpret_cast<float*>(part_h + 8 * BN);  // [2][4][BN]
  double* bE = reinterpret_cast<double*>(part_f + 8 * BN);    // [BN] best energy
  double* lE = bE + BN;                                       // [BN] last energy
  long long* bT = reinterpret_cast<long long*>(lE + BN);      // [BN] best step
  uint32_t* imp = reinterpret_cast<uint32_t*>(bT + BN);       // [2][4] improvement bits
  uint64_t* tma_bar = reinterpret_cast<uint64_t*>(imp + 8);
  uint64_t* acc_bar = tma_bar + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_bar + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n0 = (int64_t)blockIdx.x * BN;
  // (the step count comes from the host: CTAs of a large grid need not run
  // at the same time, so counters[0] may already be advanced when one starts)
  const long long t0 = R.t0;
  const int64_t K = R.steps;
  if (threadIdx.x == 0) {
    tc::mbar_init(tma_bar, 1);
    tc::mbar_init(acc_bar, 1);
    tc::fence_barrier_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, kTmemCols);
    tc::fence_before_sync();
  }
  // spin buffers start at 0 (rows past B, columns past n stay 0)
  for (size_t o = threadIdx.x * 16; o < 2 * kSbuf; o += (size_t)blockDim.x * 16)
    *reinterpret_cast<uint4*>(Ssm + o) = make_uint4(0, 0, 0, 0);
  for (int b = threadIdx.x; b < BN; b += blockDim.x) {
    const int64_t gb = n0 + b;
    const bool ok = gb < P.B;
    bE[b] = ok ? R.best_E[gb] : 0.0;
    lE[b] = ok ? R.last_E[gb] : 0.0;
    bT[b] = ok ? R.best_t[gb] : 0;
  }
  tc::fence_proxy_async_shared();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem_base = *tmem_slot;
  if (threadIdx.x == 0) {
    // all of J (every plane and k-block) and S_{t0+1} of this block of restarts
    tc::mbar_expect_tx(tma_bar, (uint32_t)nkt * Lay::kA + (uint32_t)nk * Lay::kSk);
    // (tile kt: plane kt % planes of k-block kt / planes, the MMAs' order)
    for (int kt = 0; kt < nkt; ++kt) {
      const int plane = kt % P.planes, kb = kt / P.planes;
      const CUtensorMap* ma = plane == 0 ? &tmA0 : (plane == 1 ? &tmA1 : &tmA2);
      tc::tma_load_2d(Jsm + (size_t)kt * Lay::kA, ma, tma_bar, kb * kBK, 0);
    }
    for (int kb = 0; kb < nk; ++kb)
      tc::tma_load_2d(Ssm + (size_t)kb * Lay::kSk, &tmB, tma_bar, kb * kBK, (int)n0);
  }
  // epilogue lanes: row i, quarter q, column part
  const int q = warp & 3;
  const int part = (warp - 1) >> 2;
  const int64_t i = 32 * q + lane;
  const bool epi = warp >= 1;
  const bool row_ok = epi && i < P.n;
  const uint32_t lane_off = (uint32_t)(32 * q) << 16;
  const uint32_t t_acc = tmem_base + lane_off + (uint32_t)(part * kCols);
  const uint32_t t_th = t_acc + BN, t_m = t_acc + 2 * BN, t_v = t_acc + 3 * BN;
  float h = 0.f, rs = 1.f;
  int hi = 0;
  if (row_ok) {
    h = P.hf[i];
    hi = P.hint[i];
    if (P.rowscale) rs = P.rowscale[i];
  }
  const float chh = P.k.ch * h;
  const float hm_pos = fmaf(P.k.ch, h, -P.k.mu), hm_neg = fmaf(P.k.ch, h, P.k.mu);
  if (epi) {
    // state of this warp's columns into tensor memory
#pragma unroll 1
    for (int c0 = 0; c0 < kCols; c0 += kChunk) {
      uint32_t a[kChunk], bm[kChunk], c[kChunk];
#pragma unroll
      for (int j = 0; j < kChunk; ++j) {
        const int64_t b = n0 + part * kCols + c0 + j;
        const bool ok = row_ok && b < P.B;
        const int64_t idx = b * P.ld + i;
        a[j] = __float_as_uint(ok ? P.theta[idx] : 0.f);
        bm[j] = __float_as_uint(ok ? P.m[idx] : 0.f);
        c[j] = __float_as_uint(ok ? P.v[idx] : 0.f);
      }
      tc::tmem_st8(t_th + c0, a);
      tc::tmem_st8(t_m + c0, bm);
      tc::tmem_st8(t_v + c0, c);
    }
    tc::tmem_wait_st();
  }
  int ok = tc::mbar_wait(tma_bar, 0, nullptr, kWaitCycles) ? 1 : 0;
  tc::fence_before_sync();
  ok = __syncthreads_and(ok);
  tc::fence_after_sync();
  const bool loaded = ok != 0;

  // Energies and bests of step index e (E_{t0+e+1}) from partial slot e mod 2,
  // one lane per restart (sums in track_kernel's order over the four lane
  // quarters); the improvement bits go to imp[e mod 2]. Warp 0 runs this for
  // step s - 1 while the tensor cores run step s.
  auto track = [&](int64_t e) {
    const int slot = (int)(e & 1);
    const int* pq = part_q + slot * 4 * BN;
    const int* ph = part_h + slot * 4 * BN;
    const float* pf = part_f + slot * 4 * BN;
#pragma unroll
    for (int w = 0; w < kWords; ++w) {
      const int b = 32 * w + lane;
      double E;
      if (INT_E) {
        const long long qs = (long long)pq[b] + pq[2 * BN + b] + pq[BN + b] + pq[3 * BN + b];
        const long long hs = (long long)ph[b] + ph[2 * BN + b] + ph[BN + b] + ph[3 * BN + b];
        E = R.cq * (double)qs + R.chs * (double)hs;
      } else {
        E = ((0.0 + (double)pf[b]) + (0.0 + (double)pf[2 * BN + b])) +
            ((0.0 + (double)pf[BN + b]) + (0.0 + (double)pf[3 * BN + b]));
      }
      const bool better = E < bE[b] && n0 + b < P.B;
      lE[b] = E;
      if (better) {
        bE[b] = E;
        bT[b] = t0 + e + 1;
      }
      const uint32_t bits = __ballot_sync(0xffffffffu, better);
      if (lane == 0) imp[slot * 4 + w] = bits;
    }
  };
  // This thread's columns of an improvement word of slot e mod 2.
  auto imp_mask = [&](int64_t e) -> uint32_t {
    const int c = part * kCols;
    const uint32_t w = imp[(int)(e & 1) * 4 + (c >> 5)];
    return kCols == 32 ? w : (w >> (c & 31)) & ((1u << (kCols & 31)) - 1u);
  };
  // spins consumed at steps s - 1 and s - 2 (bit c = column part * kCols + c),
  // the best spins of each column, and which columns improved in this launch
  uint32_t prev_bits = 0, prev2_bits = 0, best_bits = 0, any_bits = 0;
  float2 bc = make_float2(0.f, 0.f);
  if (epi && K > 0) bc = P.bias[t0 + 1];
  const uint32_t idesc = op_idesc(BN, FP8, P.f16);
  int64_t s = 0;
  for (; s < K && ok; ++s) {
    const long long t = t0 + s + 1;
    const int cur = (int)(s & 1);
    uint8_t* Scur = Ssm + (size_t)cur * kSbuf;
    uint8_t* Snxt = Ssm + (size_t)(cur ^ 1) * kSbuf;
    const bool last = s + 1 == K;
    int wok = 1;
    if (warp == 0) {
      if (lane == 0) {
        for (int kt = 0; kt < nkt; ++kt) {
          const int kb = kt / P.planes;
          // descriptors of the tiles; K step k adds 32 bytes (2 in the >> 4 address field)
          const uint64_t da = tc::desc_k_sw128(tc::smem_u32(Jsm + (size_t)kt * Lay::kA));
          const uint64_t db = tc::desc_k_sw128(tc::smem_u32(Scur + (size_t)kb * Lay::kSk));
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (FP8)
              tc::mma_f8(tmem_base, da + 2u * k, db + 2u * k,
                         idesc, (kt > 0 || k > 0) ? 1u : 0u);
            else
              tc::mma_f16(tmem_base, da + 2u * k, db + 2u * k,
                          idesc, (kt > 0 || k > 0) ? 1u : 0u);
          }
        }
        tc::mma_commit(acc_bar);
      }
      __syncwarp();
      if (s >= 1) track(s - 1);
    } else {
      const float2 bcs = bc;
      if (!last) bc = P.bias[t + 1];  // used by the next step
      if (s >= 2) {
        // the bests of step s - 2 are known now
        const uint32_t mk = imp_mask(s - 2);
        best_bits = (best_bits & ~mk) | (prev2_bits & mk);
        any_bits |= mk;
      }
      wok = tc::mbar_wait(acc_bar, (uint32_t)(s & 1), nullptr, kWaitCycles) ? 1 : 0;
      tc::fence_after_sync();
      uint32_t cur_bits = 0;
      if (wok) {
        int* pq = part_q + cur * 4 * BN;
        int* ph = part_h + cur * 4 * BN;
        float* pf = part_f + cur * 4 * BN;
#pragma unroll 1
        for (int c0 = 0; c0 < kCols; c0 += kChunk) {
          uint32_t r[kChunk], th[kChunk], mm[kChunk], vv[kChunk];
          tc::tmem_ld8(t_acc + c0, r);
          tc::tmem_ld8(t_th + c0, th);
          tc::tmem_ld8(t_m + c0, mm);
          tc::tmem_ld8(t_v + c0, vv);
          tc::tmem_wait_ld();
          int eq[kChunk];
          float ef[kChunk];
          uint32_t pos_bits = 0;
#pragma unroll
          for (int j = 0; j < kChunk; ++j) {
            float tj = __uint_as_float(th[j]), mj = __uint_as_float(mm[j]), vj = __uint_as_float(vv[j]);
            const float G = __uint_as_float(r[j]) * rs;
            const bool pos = sin_nonneg(tj);  // the spin this step consumed
            pos_bits |= (pos ? 1u : 0u) << j;
            if (INT_E) eq[j] = __float_as_int(__fadd_rn(pos ? G : -G, 12582912.0f));
            else ef[j] = (pos ? 1.f : -1.f) * fmaf(P.k.cq, G, chh);
            const float F = fmaf(P.k.cq, G, pos ? hm_pos : hm_neg);
            const float g = cos_proj(tj) * F;
            tj = adam_update(P.k, bcs.x, bcs.y, g, tj, mj, vj);
            th[j] = __float_as_uint(tj);
            mm[j] = __float_as_uint(mj);
            vv[j] = __float_as_uint(vj);
          }
          cur_bits |= pos_bits << c0;
          if (!last) {
            tc::tmem_st8(t_th + c0, th);
            tc::tmem_st8(t_m + c0, mm);
            tc::tmem_st8(t_v + c0, vv);
          }
          const int bl0 = part * kCols + c0;  // local restart of column j = 0
          if (row_ok) {
            const int kb = (int)(i / kBK), kk = (int)(i % kBK);
#pragma unroll
            for (int j = 0; j < kChunk; ++j) {
              const float tj = __uint_as_float(th[j]);
              const bool sp = sin_nonneg(tj);
              uint8_t* dst = Snxt + (size_t)kb * Lay::kSk + swz_offset(bl0 + j, kk, esize);
              if (FP8) *dst = sp ? 0x38 : 0xB8;
              else *reinterpret_cast<uint16_t*>(dst) = pm1_16(sp, P.f16);
              const int64_t b = n0 + bl0 + j;
              if (last && b < P.B) {
                const int64_t idx = b * P.ld + i;
                P.theta[idx] = tj;
                P.m[idx] = __uint_as_float(mm[j]);
                P.v[idx] = __uint_as_float(vv[j]);
              }
            }
          }
          if (INT_E) {
            int qv = 0, hv = 0;
#pragma unroll
            for (int j = 0; j < kChunk; ++j) {
              const unsigned int sum = __reduce_add_sync(0xffffffffu, (unsigned int)eq[j]);
              if (lane == j) qv = (int)(sum - 32u * 0x4B400000u);
            }
            if (P.has_h) {
#pragma unroll
              for (int j = 0; j < kChunk; ++j) {
                const int sum = __reduce_add_sync(0xffffffffu, ((pos_bits >> j) & 1u) ? hi : -hi);
                if (lane == j) hv = sum;
              }
            }
            if (lane < kChunk) {
              pq[q * BN + bl0 + lane] = qv;
              ph[q * BN + bl0 + lane] = hv;
            }
          } else {
            const float te = column_sums8(ef, lane);
            if ((lane & 3) == 0) pf[q * BN + bl0 + column_of_lane(lane)] = te;
          }
        }
        tc::tmem_wait_st();
      }
      prev2_bits = prev_bits;
      prev_bits = cur_bits;
    }
    // the new spins are operands of the next MMAs; partials are complete
    tc::fence_proxy_async_shared();
    tc::fence_before_sync();
    ok = __syncthreads_and(wok);
    tc::fence_after_sync();
  }
  if (ok && K > 0) {
    // the last step's energies, then the bests of the last two steps
    if (warp == 0) track(K - 1);
    __syncthreads();
    if (epi) {
      if (K >= 2) {
        const uint32_t mk = imp_mask(K - 2);
        best_bits = (best_bits & ~mk) | (prev2_bits & mk);
        any_bits |= mk;
      }
      const uint32_t mk = imp_mask(K - 1);
      best_bits = (best_bits & ~mk) | (prev_bits & mk);
      any_bits |= mk;
      if (row_ok) {
        for (int c = 0; c < kCols; ++c) {
          const int64_t b = n0 + part * kCols + c;
          if ((any_bits >> c) & 1u) R.best_s[b * R.bs_ld + i] = ((best_bits >> c) & 1u) ? 1 : -1;
        }
      }
    }
  }
  // S_{t0+K+1} to its global slot, bests back to global, step counter
  if (ok) {
    uint8_t* Sfin = Ssm + (size_t)(K & 1) * kSbuf;
    for (int64_t e = threadIdx.x; e < (int64_t)BN * P.n; e += blockDim.x) {
      const int b = (int)(e / P.n), ii = (int)(e % P.n);
      if (n0 + b >= P.B) continue;
      const uint8_t* src = Sfin + (size_t)(ii / kBK) * Lay::kSk + swz_offset(b, ii % kBK, esize);
      const int64_t idx = (n0 + b) * P.ld + ii;
      if (FP8) static_cast<uint8_t*>(R.spins_out)[idx] = *src;
      else static_cast<uint16_t*>(R.spins_out)[idx] = *reinterpret_cast<const uint16_t*>(src);
    }
    for (int b = threadIdx.x; b < BN; b += blockDim.x) {
      const int64_t gb = n0 + b;
      if (gb >= P.B) continue;
      R.best_E[gb] = bE[b];
      R.best_t[gb] = bT[b];
      R.last_E[gb] = lE[b];
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) const_cast<long long*>(P.counters)[0] = t0 + K;
  } else if (threadIdx.x == 0) {
    atomicExch(P.err, 5);
    // copies and MMAs already issued must land before the CTA frees its memory
    if (!loaded) tc::mbar_wait(tma_bar, 0, nullptr, kWaitCycles / 8);
    else if (s < K) tc::mbar_wait(acc_bar, (uint32_t)(s & 1), nullptr, kWaitCycles / 8);
  }
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem_base, kTmemCols);
  }
}

struct TcState {
  CUtensorMap A[3];
  CUtensorMap B[3];   // one per spin slot, boxes of BN restarts (streaming kernel)
  CUtensorMap Bg[3];  // one per spin slot, boxes of one restart group (resident kernel)
  // resident kernel: views of J (per plane) and of the spin slots as
  // [k-block][row][128 B] with boxes of two whole k-blocks
  CUtensorMap J2[3], S2[3];
  CUtensorMap SP[3];  // streaming kernel: the spin slots' pair views, boxes of BN restarts
  CUtensorMap Bh[3];  // pair tiles: the spin slots, boxes of BN / 2 restarts
  bool pair = false;  // streaming kernel over clusters of two CTAs sharing spin tiles
  bool split = false; // ... whose MMAs run as one per pair (cta_group::2)
  int nfull = 0;      // k-blocks lying wholly below column n (0 in the small form)
  CUtensorMap Bx[2];  // relaxed mode: one per slot of x = sin(theta), boxes of BN restarts
  int BN = 128;
  size_t smem = 0;
  int grid = 1;
  bool maps_ready = false;
  bool fp8 = false;
  bool f16 = false;       // 16-bit operands are FP16 (two-plane form), else BF16
  bool resident = false;  // one tile per CTA, state kept in tensor memory
  DevMem gsync;           // abort word + per-column barrier counters
  int emode = 0;          // resident epilogue's integer energy mode (0 F2I, 1 offset, 2 packed)
  int gn = 64;            // resident forms: restarts per group (two per CTA; small form: one)
  bool small = false;     // small form (n <= 128): all of J per CTA, spins kept on chip
  size_t small_bytes = 0;
  int small_grid = 0;     // small form: CTAs (one per block of gn restarts)
  int jres = 0, nst = 0;  // resident form: J tiles kept in shared memory, stages
  uint32_t bars = 0;      // resident form: offset of the barrier block
  size_t res_bytes = 0;   // resident form: dynamic shared memory
  DevMem err;
  DevMem trace;  // grid x 8 timestamps of the last profiled launch
};

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2D BF16 map over rows x cols (cols contiguous, row pitch ld elements), box
// of box_cols x box_rows with the 128-byte swizzle; out-of-range reads are 0.
int make_map(ising_ctx* ctx, CUtensorMap* map, const void* base, int64_t cols, int64_t rows,
             int64_t ld, int box_cols, int box_rows, bool fp8) {
  auto fn = encode_fn();
  if (!fn) return fail(ctx, ISING_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * (fp8 ? 1 : 2))};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  const_cast<void*>(base), dims,
                  strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, ISING_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return ISING_OK;
}

// View of a [rows][ld] operand as (128-byte column chunk, row, k-block) over
// its first `nfull` whole k-blocks, with boxes of two k-blocks: one copy then
// fills two consecutive k-block tiles of a stage (the k-block stride is 128
// bytes, so a box never reaches past column nfull * 128 bytes, all below n).
int make_map_pairs(ising_ctx* ctx, CUtensorMap* map, const void* base, int64_t nfull, int64_t rows,
                   int64_t ld, int box_rows, bool fp8) {
  auto fn = encode_fn();
  if (!fn) return fail(ctx, ISING_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  const int es = fp8 ? 1 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)(kRowBytes / es), (cuuint64_t)rows, (cuuint64_t)nfull};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * es), (cuuint64_t)kRowBytes};
  cuuint32_t box[3] = {(cuuint32_t)(kRowBytes / es), (cuuint32_t)box_rows, 2};
  cuuint32_t est[3] = {1, 1, 1};
  CUresult r = fn(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                  const_cast<void*>(base), dims, strides, box, est, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, ISING_ECUDA, "cuTensorMapEncodeTiled (pairs) failed (%d)", (int)r);
  return ISING_OK;
}

template <int BN, int MODE, bool INT_E, bool FP8>
int launch_bn(ising_ds* ds, TcState* st, const TcArgs& a, const CUtensorMap& mB,
              const CUtensorMap& mS2, const CUtensorMap& mBh) {
  const size_t smem = TcLayout<BN>::kBytes;
  if constexpr (BN >= 192) {
    if (st->pair && st->split) {
      auto kern = tc_step_split_kernel<BN, MODE, INT_E, FP8>;
      const size_t ssmem = TcLayout<BN, true>::kBytes;
      static bool attr_set = false;  // per instantiation
      if (!attr_set) {
        ISING_CUDA(ds->ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)ssmem));
        attr_set = true;
      }
      const int pairs = (a.mtiles + 1) / 2 * a.ntiles;
      const int clusters = std::max(1, std::min(pairs, ds->ctx->sm_count / 2));
      kern<<<2 * clusters, kThreads, ssmem, ds->ctx->stream>>>(st->A[0], st->A[1], st->A[2], mBh,
                                                               st->J2[0], st->J2[1], st->J2[2],
                                                               mS2, a);
      ISING_CUDA(ds->ctx, cudaGetLastError());
      return ISING_OK;
    }
    if (st->pair) {
      auto kern = tc_step_pair_kernel<BN, MODE, INT_E, FP8>;
      static bool attr_set = false;  // per instantiation
      if (!attr_set) {
        ISING_CUDA(ds->ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem));
        attr_set = true;
      }
      // one cluster of two CTAs per pair of SMs, at most one per pair tile
      const int pairs = (a.mtiles + 1) / 2 * a.ntiles;
      const int clusters = std::max(1, std::min(pairs, ds->ctx->sm_count / 2));
      kern<<<2 * clusters, kThreads, smem, ds->ctx->stream>>>(st->A[0], st->A[1], st->A[2], mBh,
                                                              st->J2[0], st->J2[1], st->J2[2],
                                                              mS2, a);
      ISING_CUDA(ds->ctx, cudaGetLastError());
      return ISING_OK;
    }
  }
  auto kern = tc_step_kernel<BN, MODE, INT_E, FP8>;
  static bool attr_set = false;  // per instantiation
  if (!attr_set) {
    ISING_CUDA(ds->ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
    attr_set = true;
  }
  kern<<<st->grid, kThreads, smem, ds->ctx->stream>>>(st->A[0], st->A[1], st->A[2], mB, st->J2[0],
                                                       st->J2[1], st->J2[2], mS2, a);
  ISING_CUDA(ds->ctx, cudaGetLastError());
  return ISING_OK;
}

template <int MODE, bool INT_E, bool FP8>
int launch_bn_sel(ising_ds* ds, TcState* st, const TcArgs& a, const CUtensorMap& mB,
                  const CUtensorMap& mS2, const CUtensorMap& mBh) {
  switch (st->BN) {
    case 256: return launch_bn<256, MODE, INT_E, FP8>(ds, st, a, mB, mS2, mBh);
    case 224: return launch_bn<224, MODE, INT_E, FP8>(ds, st, a, mB, mS2, mBh);
    case 64: return launch_bn<64, MODE, INT_E, FP8>(ds, st, a, mB, mS2, mBh);
    default: return launch_bn<128, MODE, INT_E, FP8>(ds, st, a, mB, mS2, mBh);
  }
}

template <int MODE, bool INT_E>
int launch_mode(ising_ds* ds, TcState* st, const TcArgs& a, const CUtensorMap& mB,
                const CUtensorMap& mS2, const CUtensorMap& mBh) {
  return st->fp8 ? launch_bn_sel<MODE, INT_E, true>(ds, st, a, mB, mS2, mBh)
                 : launch_bn_sel<MODE, INT_E, false>(ds, st, a, mB, mS2, mBh);
}

// Relaxed-product update: 16-bit operands only (x in E4M3 would be too
// coarse); never in pairs (the relaxed spins have no half-box maps).
template <bool INT_E>
int launch_relaxed(ising_ds* ds, TcState* st, const TcArgs& a, const CUtensorMap& mB,
                   const CUtensorMap& mS2) {
  if (st->fp8) return fail(ds->ctx, ISING_ENOTSUP, "relaxed product needs BF16 operands");
  return launch_bn_sel<kModeRelaxed, INT_E, false>(ds, st, a, mB, mS2, mB);
}

}  // namespace

template <int GN, bool INT_E, bool FP8>
int resident_attr(ising_ctx* ctx, size_t smem, int* blocks_per_sm) {
  auto kern = tc_resident_kernel<GN, INT_E, FP8>;
  ISING_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ISING_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, kThreads, smem));
  return ISING_OK;
}

template <int GN, bool INT_E, bool FP8>
int resident_launch(ising_ds* ds, TcState* st, const TcResArgs& ra) {
  auto kern = tc_resident_kernel<GN, INT_E, FP8>;
  void* args[] = {&st->A[0],  &st->A[1],  &st->A[2],  &st->Bg[0], &st->Bg[1], &st->Bg[2],
                  &st->J2[0], &st->J2[1], &st->J2[2], &st->S2[0], &st->S2[1], &st->S2[2],
                  const_cast<TcResArgs*>(&ra)};
  ISING_CUDA(ds->ctx, cudaLaunchCooperativeKernel((const void*)kern, dim3(st->grid), dim3(kThreads),
                                                  args, st->res_bytes, ds->ctx->stream));
  return ISING_OK;
}

template <int GN>
int resident_attr_bn(ising_ds* ds, bool fp8, size_t smem, int* nb) {
  if (ds->int_energy)
    return fp8 ? resident_attr<GN, true, true>(ds->ctx, smem, nb) : resident_attr<GN, true, false>(ds->ctx, smem, nb);
  return fp8 ? resident_attr<GN, false, true>(ds->ctx, smem, nb) : resident_attr<GN, false, false>(ds->ctx, smem, nb);
}

template <int BN>
int resident_launch_bn(ising_ds* ds, TcState* st, const TcResArgs& ra) {
  if (ds->int_energy)
    return st->fp8 ? resident_launch<BN, true, true>(ds, st, ra) : resident_launch<BN, true, false>(ds, st, ra);
  return st->fp8 ? resident_launch<BN, false, true>(ds, st, ra) : resident_launch<BN, false, false>(ds, st, ra);
}

template <int BN, bool INT_E, bool FP8>
int small_launch(ising_ds* ds, TcState* st, const TcSmallArgs& a) {
  auto kern = tc_small_kernel<BN, INT_E, FP8>;
  ISING_CUDA(ds->ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)st->small_bytes));
  kern<<<st->small_grid, kSmallThreads, st->small_bytes, ds->ctx->stream>>>(
      st->A[0], st->A[1], st->A[2], st->Bg[(ds->t + 1) % 3], a);
  ISING_CUDA(ds->ctx, cudaGetLastError());
  return ISING_OK;
}

template <int BN>
int small_launch_bn(ising_ds* ds, TcState* st, const TcSmallArgs& a) {
  if (ds->int_energy)
    return st->fp8 ? small_launch<BN, true, true>(ds, st, a) : small_launch<BN, true, false>(ds, st, a);
  return st->fp8 ? small_launch<BN, false, true>(ds, st, a) : small_launch<BN, false, false>(ds, st, a);
}

// Abort word, then one arrival counter per restart group of each column, 128
// bytes apart.
static size_t gsync_bytes(const ising_ds* ds, const TcState* st) {
  return (size_t)(1 + 2 * ceil_div_i(ds->B, st->BN)) * 128;
}

int tc_setup(ising_ds* ds) {
  ising_ctx* ctx = ds->ctx;
  const DevInstance& I = ds->inst;
  if (ctx->smem_optin < TcLayout<256>::kBytes)
    return fail(ctx, ISING_ENOTSUP, "device lacks the shared memory the tensor-core step needs");
  auto st = new TcState();
  ds->tc = st;
  const bool exact16 = I.j_integer && I.j_absmax <= 16.0;
  const bool exact256 = I.j_integer && I.j_absmax <= 256.0;
  if (ds->relaxed()) {
    // x = sin(theta) goes to the tensor cores in BF16, so J does too
    if (ds->prec == ISING_PREC_FP8)
      return fail(ctx, ISING_ENOTSUP, "relaxed product: E4M3 is too coarse for x; use BF16");
    if (ds->prec == ISING_PREC_AUTO) ds->prec = ISING_PREC_TC;
  }
  // AUTO: E4M3 when it holds J exactly, else the exact BF16 form
  if (ds->prec == ISING_PREC_AUTO) ds->prec = exact16 ? ISING_PREC_FP8 : ISING_PREC_TC;
  st->fp8 = ds->prec == ISING_PREC_FP8;
  ds->ld = st->fp8 ? (ds->n + 15) / 16 * 16 : (ds->n + 7) / 8 * 8;
  ds->Bp = ds->B;
  ds->spin_kind = st->fp8 ? kSpinE4M3 : kSpinBF16;
  ds->mtiles = 4 * ceil_div_i(ds->n, kBM);  // one energy-partial row per epilogue lane quarter
  st->BN = ds->B <= 64 ? 64 : (ds->B >= 2048 ? 256 : 128);
  if (st->BN == 256) {
    // tiles of 224 restarts when they fill the SMs' waves better: the
    // busiest SM's share, waves x BN, sets the step time
    auto cost = [&](int bn) {
      const int64_t tiles = (int64_t)ceil_div_i(ds->n, kBM) * ceil_div_i(ds->B, bn);
      return (tiles + ctx->sm_count - 1) / ctx->sm_count * bn;
    };
    if (cost(224) < cost(256)) st->BN = 224;
  }
  const int64_t plane_elems = ds->n * ds->ld;
  int g = (int)std::min<int64_t>((plane_elems + 255) / 256, (int64_t)ctx->sm_count * 16);
  if (st->fp8) {
    ds->planes = 1;
    ISING_TRY(dev_alloc(ctx, ds->Jop[0], plane_elems));
    const float* rs = nullptr;
    if (!exact16) {
      // J / scale_i rounded to E4M3: the products are no longer integers
      ds->int_energy = false;
      ISING_TRY(dev_alloc(ctx, ds->rowscale, ds->n * 4));
      row_absmax_kernel<<<(int)std::min<int64_t>(ds->n, 65535), 256, 0, ctx->stream>>>(
          I.J.p, I.j_dtype, ds->n, ds->rowscale.as<float>());
      rs = ds->rowscale.as<float>();
    }
    to_fp8_kernel<<<g, 256, 0, ctx->stream>>>(I.J.p, I.j_dtype, ds->n, ds->ld, rs,
                                              ds->Jop[0].as<uint8_t>());
    ISING_CUDA(ctx, cudaGetLastError());
    for (int p = 0; p < 3; ++p)
      ISING_TRY(make_map(ctx, &st->A[p], ds->Jop[0].p, ds->n, ds->n, ds->ld, 128, kBM, true));
  } else if (exact256 || ds->prec == ISING_PREC_BF16) {
    // one BF16 plane: exact for integers up to 256; beyond that it rounds J,
    // and the sums are no longer the instance's integers
    ds->planes = 1;
    if (!exact256) ds->int_energy = false;
    ISING_TRY(dev_alloc(ctx, ds->Jop[0], plane_elems * 2));
    to_planes_kernel<<<g, 256, 0, ctx->stream>>>(I.J.p, I.j_dtype, ds->n, ds->ld, 0, 1, nullptr,
                                                 ds->Jop[0].as<uint16_t>(), nullptr);
    ISING_CUDA(ctx, cudaGetLastError());
    for (int p = 0; p < 3; ++p)
      ISING_TRY(make_map(ctx, &st->A[p], ds->Jop[0].p, ds->n, ds->n, ds->ld, 64, kBM, false));
  } else {
    // FP16 planes: integers up to 2048 in one plane and up to 65504 in two
    // (hi + lo, both exact); other J as hi + lo of J_ij / scale_i with a
    // power-of-two scale per row (about 22 significant bits; the products are
    // then no longer integers)
    st->f16 = true;
    ds->spin_kind = kSpinF16;
    const bool int2048 = I.j_integer && I.j_absmax <= 2048.0;
    const bool int65504 = I.j_integer && I.j_absmax <= 65504.0;
    ds->planes = int2048 ? 1 : 2;
    const float* rs = nullptr;
    if (!int65504) {
      ds->int_energy = false;
      ISING_TRY(dev_alloc(ctx, ds->rowscale, ds->n * 4));
      row_pow2_scale_kernel<<<(int)std::min<int64_t>(ds->n, 65535), 256, 0, ctx->stream>>>(
          I.J.p, I.j_dtype, ds->n, ds->rowscale.as<float>());
      ISING_CUDA(ctx, cudaGetLastError());
      rs = ds->rowscale.as<float>();
    }
    for (int p = 0; p < ds->planes; ++p) ISING_TRY(dev_alloc(ctx, ds->Jop[p], plane_elems * 2));
    to_planes_kernel<<<g, 256, 0, ctx->stream>>>(
        I.J.p, I.j_dtype, ds->n, ds->ld, 1, ds->planes, rs, ds->Jop[0].as<uint16_t>(),
        ds->planes == 2 ? ds->Jop[1].as<uint16_t>() : nullptr);
    ISING_CUDA(ctx, cudaGetLastError());
    for (int p = 0; p < 3; ++p) {
      const void* base = ds->Jop[p < ds->planes ? p : 0].p;
      ISING_TRY(make_map(ctx, &st->A[p], base, ds->n, ds->n, ds->ld, 64, kBM, false));
    }
  }
  ISING_TRY(dev_alloc(ctx, st->err, 16));
  ISING_CUDA(ctx, cudaMemsetAsync(st->err.p, 0, 16, ctx->stream));
  if (ds->int_energy) {
    // |G_i| < 2^22 holds for integer energies; pairs of column sums fit one
    // 32-bit reduction when 32 max_i sum_j |J_ij| < 2^15
    st->emode = 1;
    if (I.layout == ISING_LAYOUT_DENSE) {
      DevMem mx;
      ISING_TRY(dev_alloc(ctx, mx, 8));
      ISING_CUDA(ctx, cudaMemsetAsync(mx.p, 0, 8, ctx->stream));
      const int rg = (int)std::max<int64_t>(1, std::min<int64_t>((ds->n + 7) / 8, (int64_t)ctx->sm_count * 16));
      row_abssum_max_kernel<<<rg, 256, 0, ctx->stream>>>(I.J.p, I.j_dtype, ds->n, mx.as<unsigned long long>());
      ISING_CUDA(ctx, cudaGetLastError());
      unsigned long long r = 0;
      ISING_CUDA(ctx, cudaMemcpyAsync(&r, mx.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
      ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      if (32ull * r < 32768ull) st->emode = 2;
    }
  }
  st->nfull = (int)(ds->n / (st->fp8 ? 128 : 64));
  // resident form when every (128 x 2 GN) tile gets its own co-resident CTA
  // (a tensor-memory kernel holds its SM alone): two groups of GN restarts
  // per CTA, 64 each, or 32 when B <= 64
  // small form: n <= 128, every CTA self-contained (no co-residency needed);
  // the narrowest block of restarts (32, 64 or 128) that still fits one wave
  if (!(ds->p.flags & (ISING_DS_STREAMING | ISING_DS_CONVERGE)) && !ds->relaxed() && ds->n <= kBM) {
    int bn = 128;
    for (int c : {32, 64})
      if (ceil_div_i(ds->B, c) <= ctx->sm_count) {
        bn = c;
        break;
      }
    const int nk = ceil_div_i(ds->n, st->fp8 ? 128 : 64), nkt = nk * ds->planes;
    const size_t bytes = (size_t)nkt * kBM * kRowBytes + 2 * (size_t)nk * bn * kRowBytes +
                         (size_t)bn * (2 * 3 * 4 * 4 + 8 + 8 + 8) + 32 + 64 + 1024;
    if (bytes <= (size_t)ctx->smem_optin) {
      st->small = true;
      st->resident = true;
      st->nfull = 0;
      st->gn = bn;
      st->small_grid = ceil_div_i(ds->B, bn);
      st->small_bytes = bytes;
    }
  }
  if (!st->resident && !(ds->p.flags & ISING_DS_STREAMING) && !ds->relaxed()) {
    const int gn = ds->B > 64 ? 64 : 32;
    const int tiles = ceil_div_i(ds->n, kBM) * ceil_div_i(ds->B, 2 * gn);
    // shared memory: resident J tiles (as many as leave room for 4 stages of 2 k-blocks),
    // then the stages, then the barrier block
    const int64_t kA = (int64_t)kBM * kRowBytes, kStage = 2 * (kA + (int64_t)gn * kRowBytes);
    const int64_t region = ((int64_t)ctx->smem_optin - 1024 - 512) / 1024 * 1024;
    const int nkt = ceil_div_i(ds->n, st->fp8 ? 128 : 64) * ds->planes;
    const int jres = (int)std::min<int64_t>(nkt, std::max<int64_t>(0, (region - 4 * kStage) / kA));
    const int nst = (int)std::min<int64_t>(8, (region - jres * kA) / kStage);
    int nb = 0;
    if (nst >= 2) {
      const size_t bytes = (size_t)region + 512 + 1024;
      ISING_TRY(gn == 64 ? resident_attr_bn<64>(ds, st->fp8, bytes, &nb)
                         : resident_attr_bn<32>(ds, st->fp8, bytes, &nb));
      if (nb >= 1 && tiles <= nb * ctx->sm_count) {
        st->resident = true;
        st->BN = 2 * gn;
        st->gn = gn;
        st->grid = tiles;
        st->jres = jres;
        st->nst = nst;
        st->bars = (uint32_t)region;
        st->res_bytes = bytes;
      }
    }
  }
  if (st->resident && !st->small) {
    ISING_TRY(dev_alloc(ctx, st->gsync, gsync_bytes(ds, st)));
  } else {
    // streaming launches (and, in the small form, the final evaluation)
    const int tiles = ceil_div_i(ds->n, kBM) * ceil_div_i(ds->B, st->BN);
    st->grid = std::max(1, std::min(tiles, ctx->sm_count));
  }
  return ISING_OK;
}

// The B-operand maps point at the spin buffers, which exist only after the
// common allocation; they are built on first use.
static int tc_maps(ising_ds* ds, TcState* st) {
  static_assert(sizeof(CUtensorMap) == 128, "CUtensorMap size");
  for (int s = 0; s < 3; ++s) {
    ISING_TRY(make_map(ds->ctx, &st->B[s], ds->spins[s].p, ds->n, ds->B, ds->ld,
                       st->fp8 ? 128 : 64, st->BN, st->fp8));
    if (st->nfull >= 2) {
      ISING_TRY(make_map_pairs(ds->ctx, &st->SP[s], ds->spins[s].p, st->nfull, ds->B, ds->ld, st->BN,
                               st->fp8));
      if (st->resident)
        ISING_TRY(make_map_pairs(ds->ctx, &st->S2[s], ds->spins[s].p, st->nfull, ds->B, ds->ld,
                                 st->gn, st->fp8));
    }
    if (st->resident)
      ISING_TRY(make_map(ds->ctx, &st->Bg[s], ds->spins[s].p, ds->n, ds->B, ds->ld,
                         st->fp8 ? 128 : 64, st->gn, st->fp8));
    if (st->pair)
      ISING_TRY(make_map(ds->ctx, &st->Bh[s], ds->spins[s].p, ds->n, ds->B, ds->ld,
                         st->fp8 ? 128 : 64, st->BN / 2, st->fp8));
  }
  if (st->nfull >= 2)
    for (int p = 0; p < 3; ++p)
      ISING_TRY(make_map_pairs(ds->ctx, &st->J2[p], ds->Jop[p < ds->planes ? p : 0].p, st->nfull,
                               ds->n, ds->ld, kBM, st->fp8));
  if (ds->relaxed())
    for (int s = 0; s < 2; ++s)
      ISING_TRY(make_map(ds->ctx, &st->Bx[s], ds->xbuf[s].p, ds->n, ds->B, ds->ld, 64, st->BN, false));
  return ISING_OK;
}

int tc_run(ising_ds* ds, int mode, float* Gout) {
  auto st = static_cast<TcState*>(ds->tc);
  if (!st->maps_ready) {
    ISING_TRY(tc_maps(ds, st));
    st->maps_ready = true;
  }
  const int64_t t = ds->t + 1;
  const int ps = (int)(t % 2);
  TcArgs a;
  a.n = ds->n;
  a.B = ds->B;
  a.ld = ds->ld;
  a.nk = ceil_div_i(ds->n, st->fp8 ? 128 : 64);
  a.planes = ds->planes;
  a.f16 = st->f16 ? 1 : 0;
  a.mtiles = ceil_div_i(ds->n, kBM);
  a.ntiles = ceil_div_i(ds->B, st->BN);
  a.k = ds->k;
  a.bias = ds->bias.as<float2>();
  a.counters = ds->counters.as<long long>();
  a.S = ds->spins[t % 3].p;
  a.Snext = ds->spins[(t + 1) % 3].p;
  a.Xnext = ds->relaxed() ? ds->xbuf[(t + 1) % 2].p : nullptr;
  a.rowscale = ds->rowscale.p ? ds->rowscale.as<float>() : nullptr;
  a.theta = ds->theta.as<float>();
  a.m = ds->m.as<float>();
  a.v = ds->v.as<float>();
  a.hf = ds->hf.as<float>();
  a.hint = ds->hint.as<int32_t>();
  a.qpart = ds->qpart[ps].as<long long>();
  a.hpart = ds->hpart[ps].as<long long>();
  a.epart = ds->epart[ps].as<float>();
  a.Gout = Gout;
  a.err = st->err.as<int>();
  a.has_h = ds->inst.has_h ? 1 : 0;
  // |G_i| <= max |J_ij| * n in stored units
  a.gmagic = st->emode;
  a.trace = nullptr;
  a.live32 = ds->live.p ? ds->live.as<int>() : nullptr;
  a.work = ds->work.as<unsigned long long>();
  if (mode == kModeUpdate && ds->fold_track) {
    a.fold = 1;
    a.trk = track_args(ds);
  }
  if (ds->p.flags & ISING_DS_PROFILE) {
    if (!st->trace.p) ISING_TRY(dev_alloc(ds->ctx, st->trace, (size_t)st->grid * 8 * 8));
    a.trace = st->trace.as<unsigned long long>();
  }
  const CUtensorMap& mS = st->B[t % 3];
  const CUtensorMap& mS2 = st->SP[t % 3];
  const CUtensorMap& mSh = st->Bh[t % 3];
  a.nfull = st->nfull;
  const bool ie = ds->int_energy;
  switch (mode) {
    case kModeUpdate: return ie ? launch_mode<kModeUpdate, true>(ds, st, a, mS, mS2, mSh)
                                : launch_mode<kModeUpdate, false>(ds, st, a, mS, mS2, mSh);
    case kModeEnergy: return ie ? launch_mode<kModeEnergy, true>(ds, st, a, mS, mS2, mSh)
                                : launch_mode<kModeEnergy, false>(ds, st, a, mS, mS2, mSh);
    case kModeRelaxed: {
      // the product runs on x_t; the epilogue reads s_t and writes s_{t+1},
      // x_{t+1} (x has no pair view: one copy per k-block)
      const CUtensorMap& mX = st->Bx[t % 2];
      a.nfull = 0;
      return ie ? launch_relaxed<true>(ds, st, a, mX, mS2) : launch_relaxed<false>(ds, st, a, mX, mS2);
    }
    default: return launch_mode<kModeCoupling, true>(ds, st, a, mS, mS2, mSh);
  }
}

int tc_step(ising_ds* ds, int mode, float* Gout) {
  auto st = static_cast<TcState*>(ds->tc);
  if (!st->resident) return tc_run(ds, mode, Gout);
  // the streaming kernel with the resident tile shape: one CTA per tile
  return tc_run(ds, mode, Gout);
}

bool tc_is_resident(ising_ds* ds) {
  auto st = static_cast<TcState*>(ds->tc);
  return st && st->resident;
}

int tc_resident_form(ising_ds* ds) {
  auto st = static_cast<TcState*>(ds->tc);
  return !st || !st->resident ? 0 : (st->small ? 2 : 1);
}

int tc_run_resident(ising_ds* ds, int64_t steps) {
  auto st = static_cast<TcState*>(ds->tc);
  if (!st->maps_ready) {
    ISING_TRY(tc_maps(ds, st));
    st->maps_ready = true;
  }
  if (st->small) {
    TcSmallArgs sa;
    TcArgs& a = sa.P;
    a.n = ds->n;
    a.B = ds->B;
    a.ld = ds->ld;
    a.nk = ceil_div_i(ds->n, st->fp8 ? 128 : 64);
    a.planes = ds->planes;
    a.f16 = st->f16 ? 1 : 0;
    a.mtiles = 1;
    a.ntiles = st->small_grid;
    a.k = ds->k;
    a.bias = ds->bias.as<float2>();
    a.counters = ds->counters.as<long long>();
    a.S = nullptr;
    a.Snext = nullptr;
    a.Xnext = nullptr;
    a.rowscale = ds->rowscale.p ? ds->rowscale.as<float>() : nullptr;
    a.theta = ds->theta.as<float>();
    a.m = ds->m.as<float>();
    a.v = ds->v.as<float>();
    a.hf = ds->hf.as<float>();
    a.hint = ds->hint.as<int32_t>();
    a.qpart = a.hpart = nullptr;
    a.epart = nullptr;
    a.Gout = nullptr;
    a.err = st->err.as<int>();
    a.has_h = ds->inst.has_h ? 1 : 0;
    a.gmagic = st->emode;
    a.trace = nullptr;
    a.live32 = nullptr;  // the resident forms do not retire restarts
    a.work = nullptr;
    sa.steps = steps;
    sa.t0 = ds->t;
    sa.spins_out = ds->spins[(ds->t + steps + 1) % 3].p;
    sa.best_E = ds->best_E.as<double>();
    sa.best_t = ds->best_t.as<long long>();
    sa.best_s = ds->best_s.as<int8_t>();
    sa.last_E = ds->last_E.as<double>();
    sa.bs_ld = ds->bs_ld;
    sa.cq = ds->inst.cq;
    sa.chs = ds->inst.ch * std::ldexp(1.0, -ds->h_shift);
    return st->gn == 128 ? small_launch_bn<128>(ds, st, sa)
                         : (st->gn == 64 ? small_launch_bn<64>(ds, st, sa) : small_launch_bn<32>(ds, st, sa));
  }
  ISING_CUDA(ds->ctx, cudaMemsetAsync(st->gsync.p, 0, gsync_bytes(ds, st), ds->ctx->stream));
  TcResArgs r;
  TcArgs& a = r.P;
  a.n = ds->n;
  a.B = ds->B;
  a.ld = ds->ld;
  a.nk = ceil_div_i(ds->n, st->fp8 ? 128 : 64);
  a.planes = ds->planes;
  a.f16 = st->f16 ? 1 : 0;
  a.mtiles = ceil_div_i(ds->n, kBM);
  a.ntiles = ceil_div_i(ds->B, st->BN);
  a.k = ds->k;
  a.bias = ds->bias.as<float2>();
  a.counters = ds->counters.as<long long>();
  a.S = nullptr;
  a.Snext = nullptr;
  a.rowscale = ds->rowscale.p ? ds->rowscale.as<float>() : nullptr;
  a.theta = ds->theta.as<float>();
  a.m = ds->m.as<float>();
  a.v = ds->v.as<float>();
  a.hf = ds->hf.as<float>();
  a.hint = ds->hint.as<int32_t>();
  a.qpart = a.hpart = nullptr;
  a.epart = nullptr;
  a.Gout = nullptr;
  a.err = st->err.as<int>();
  a.has_h = ds->inst.has_h ? 1 : 0;
  // |G_i| <= max |J_ij| * n in stored units
  a.gmagic = st->emode;
  a.trace = nullptr;
  a.live32 = nullptr;  // the resident forms do not retire restarts
  a.work = nullptr;
  if (ds->p.flags & ISING_DS_PROFILE) {
    if (!st->trace.p) ISING_TRY(dev_alloc(ds->ctx, st->trace, (size_t)st->grid * 8 * 8));
    a.trace = st->trace.as<unsigned long long>();
  }
  r.steps = steps;
  for (int k = 0; k < 3; ++k) r.spins[k] = ds->spins[k].p;
  for (int k = 0; k < 2; ++k) {
    r.qpart[k] = ds->qpart[k].as<long long>();
    r.hpart[k] = ds->hpart[k].as<long long>();
    r.epart[k] = ds->epart[k].as<float>();
  }
  r.gabort = st->gsync.as<int>();
  r.gbar = st->gsync.as<unsigned int>() + 32;
  r.best_E = ds->best_E.as<double>();
  r.best_t = ds->best_t.as<long long>();
  r.best_s = ds->best_s.as<int8_t>();
  r.bs_ld = ds->bs_ld;
  r.last_E = ds->last_E.as<double>();
  r.cq = ds->inst.cq;
  r.chs = ds->inst.ch * std::ldexp(1.0, -ds->h_shift);
  r.rows = ds->mtiles;
  r.slice = ceil_div_i(st->gn, ceil_div_i(ds->n, kBM));
  r.jres = st->jres;
  r.T = ds->T;
  const bool conv = ds->conv.p != nullptr;
  r.conv_ring = conv ? ds->conv_ring() : nullptr;
  r.conv_init = conv ? ds->conv_init() : nullptr;
  r.conv_step = conv ? ds->conv_step() : nullptr;
  r.conv_count = conv ? ds->conv_count() : nullptr;
  r.nst = st->nst;
  r.bars = st->bars;
  r.nfull = st->nfull;
  return st->gn == 64 ? resident_launch_bn<64>(ds, st, r) : resident_launch_bn<32>(ds, st, r);
}

int tc_error(ising_ds* ds) {
  auto st = static_cast<TcState*>(ds->tc);
  if (!st) return ISING_OK;
  int e = 0;
  ISING_CUDA(ds->ctx, cudaMemcpyAsync(&e, st->err.p, 4, cudaMemcpyDeviceToHost, ds->ctx->stream));
  ISING_CUDA(ds->ctx, cudaStreamSynchronize(ds->ctx->stream));
  if (e) return fail(ds->ctx, ISING_ETIMEOUT, "tensor-core step: a bounded wait gave up (role %d)", e);
  return ISING_OK;
}

int tc_trace(ising_ds* ds, uint64_t* out, int64_t cap, int64_t* count) {
  auto st = static_cast<TcState*>(ds->tc);
  *count = 0;
  if (!st || !st->trace.p) return ISING_OK;
  const int64_t n = std::min<int64_t>(cap, (int64_t)st->grid * 8);
  if (n > 0)
    ISING_CUDA(ds->ctx, cudaMemcpyAsync(out, st->trace.p, n * 8, cudaMemcpyDeviceToHost, ds->ctx->stream));
  ISING_CUDA(ds->ctx, cudaStreamSynchronize(ds->ctx->stream));
  *count = (int64_t)st->grid * 8;
  return ISING_OK;
}

bool tc_packable(const ising_ds* ds) {
  auto st = static_cast<const TcState*>(ds->tc);
  return ds->path == ISING_PATH_TC && st && !st->resident && !ds->relaxed();
}

uint64_t tc_pack_key(const ising_ds* ds) {
  auto st = static_cast<const TcState*>(ds->tc);
  // members of one launch share the operand type, the energy mode and the
  // number of J planes (which sets the stage layout of the launch)
  return (st->fp8 ? 1u : 0u) | (ds->int_energy ? 2u : 0u) | (ds->planes == 2 ? 4u : 0u);
}

int tc_bn(const ising_ds* ds) { return static_cast<const TcState*>(ds->tc)->BN; }

int tc_tile_pair(const ising_ds* ds) {
  auto st = static_cast<const TcState*>(ds->tc);
  return st->pair ? (st->split ? 2 : 1) : 0;
}

// Restart-tile widths the streaming form can take for this session (tiles at
// least half used); none for the resident forms.
int tc_bn_candidates(const ising_ds* ds, int* out) {
  auto st = static_cast<const TcState*>(ds->tc);
  if (!st || st->resident) return 0;
  int k = 0;
  for (int bn : {64, 128, 224, 256})
    if (bn == 64 || bn / 2 < ds->B) out[k++] = bn;
  // the same wide tiles over clusters of two CTAs sharing spin tiles
  // (kTcPair: a flag on the width; with kTcSplit their MMAs run as one),
  // when there are two row tiles to pair
  if (!ds->relaxed() && ds->n > kBM)
    for (int bn : {224, 256})
      if (bn / 2 < ds->B) {
        out[k++] = bn | kTcPair;
        out[k++] = bn | kTcPair | kTcSplit;
      }
  return k;
}

// Switches the streaming form to tiles of `bn` restarts (the products, and
// so the results, do not depend on it); the operand maps are rebuilt on the
// next launch.
int tc_set_bn(ising_ds* ds, int code) {
  auto st = static_cast<TcState*>(ds->tc);
  if (st->resident) return fail(ds->ctx, ISING_EINVAL, "tile width of a resident form");
  const int bn = code & ~(kTcPair | kTcSplit);
  const bool pair = (code & kTcPair) != 0 && bn >= 192 && !ds->relaxed();
  const bool split = pair && (code & kTcSplit) != 0;
  if (st->BN == bn && st->pair == pair && st->split == split) return ISING_OK;
  st->BN = bn;
  st->pair = pair;
  st->split = split;
  st->maps_ready = false;
  st->trace.release();
  const int tiles = ceil_div_i(ds->n, kBM) * ceil_div_i(ds->B, bn);
  st->grid = std::max(1, std::min(tiles, ds->ctx->sm_count));
  return ISING_OK;
}

size_t tc_pack_entry_bytes() { return sizeof(PackEntry); }

// The session's pack entry (host copy): its maps, all spin and partial
// slots, and the arguments tc_run would pass (slot fields unused).
int tc_pack_entry(ising_ds* ds, void* host_entry) {
  auto st = static_cast<TcState*>(ds->tc);
  if (!st->maps_ready) {
    ISING_TRY(tc_maps(ds, st));
    st->maps_ready = true;
  }
  PackEntry* e = static_cast<PackEntry*>(host_entry);
  memset(e, 0, sizeof(PackEntry));
  for (int p = 0; p < 3; ++p) {
    e->A[p] = st->A[p];
    e->J2[p] = st->nfull >= 2 ? st->J2[p] : st->A[p];
    e->B[p] = st->B[p];
    e->S2[p] = st->nfull >= 2 ? st->SP[p] : st->B[p];
    e->spins[p] = ds->spins[p].p;
  }
  for (int k = 0; k < 2; ++k) {
    e->qpart[k] = ds->qpart[k].as<long long>();
    e->hpart[k] = ds->hpart[k].as<long long>();
    e->epart[k] = ds->epart[k].as<float>();
  }
  TcArgs& a = e->args;
  a.n = ds->n;
  a.B = ds->B;
  a.ld = ds->ld;
  a.nk = ceil_div_i(ds->n, st->fp8 ? 128 : 64);
  a.planes = ds->planes;
  a.f16 = st->f16 ? 1 : 0;
  a.mtiles = ceil_div_i(ds->n, kBM);
  a.ntiles = ceil_div_i(ds->B, st->BN);
  a.k = ds->k;
  a.bias = ds->bias.as<float2>();
  a.counters = ds->counters.as<long long>();
  a.rowscale = ds->rowscale.p ? ds->rowscale.as<float>() : nullptr;
  a.theta = ds->theta.as<float>();
  a.m = ds->m.as<float>();
  a.v = ds->v.as<float>();
  a.hf = ds->hf.as<float>();
  a.hint = ds->hint.as<int32_t>();
  a.err = st->err.as<int>();
  a.has_h = ds->inst.has_h ? 1 : 0;
  a.gmagic = st->emode;
  a.nfull = st->nfull;
  a.live32 = ds->live.p ? ds->live.as<int>() : nullptr;
  a.work = ds->work.as<unsigned long long>();
  return ISING_OK;
}

namespace {
template <int BN, bool INT_E, bool FP8>
int pack_launch_t(ising_ctx* ctx, const void* entries, const int* start, int count, int tiles,
                  int* err, bool planes2, const PackFold& f) {
  auto kern = tc_pack_kernel<BN, INT_E, FP8>;
  const size_t smem = TcLayout<BN>::kBytes;
  static bool attr_set = false;  // per instantiation
  if (!attr_set) {
    ISING_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set = true;
  }
  const int grid = std::max(1, std::min(tiles, ctx->sm_count));
  kern<<<grid, kThreads, smem, ctx->stream>>>(static_cast<const PackEntry*>(entries), start, count, err,
                                              planes2, f.trk, f.rstart, f.done);
  ISING_CUDA(ctx, cudaGetLastError());
  return ISING_OK;
}

template <int BN>
int pack_launch_bn(ising_ctx* ctx, bool ie, bool fp8, bool p2, const void* entries,
                   const int* start, int count, int tiles, int* err, const PackFold& f) {
  if (ie) return fp8 ? pack_launch_t<BN, true, true>(ctx, entries, start, count, tiles, err, p2, f)
                     : pack_launch_t<BN, true, false>(ctx, entries, start, count, tiles, err, p2, f);
  return fp8 ? pack_launch_t<BN, false, true>(ctx, entries, start, count, tiles, err, p2, f)
             : pack_launch_t<BN, false, false>(ctx, entries, start, count, tiles, err, p2, f);
}
}  // namespace

int tc_pack_launch(ising_ctx* ctx, uint64_t key, int bn, const void* entries, const int* start,
                   int count, int tiles, int* err, const PackFold& f) {
  const bool fp8 = key & 1u, ie = (key & 2u) != 0, p2 = (key & 4u) != 0;
  switch (bn) {
    case 256: return pack_launch_bn<256>(ctx, ie, fp8, p2, entries, start, count, tiles, err, f);
    case 224: return pack_launch_bn<224>(ctx, ie, fp8, p2, entries, start, count, tiles, err, f);
    case 128: return pack_launch_bn<128>(ctx, ie, fp8, p2, entries, start, count, tiles, err, f);
    case 64: return pack_launch_bn<64>(ctx, ie, fp8, p2, entries, start, count, tiles, err, f);
    default: return fail(ctx, ISING_EINVAL, "pack: unknown tile width");
  }
}

void tc_release(ising_ds* ds) {
  delete static_cast<TcState*>(ds->tc);
  ds->tc = nullptr;
}

}  // namespace ising
