// K1: pruning (Sec. III-A, Algorithm 1) and K5: reconstruction.
//
// Round-synchronous: every decision of round r is taken from the state at the
// start of the step that makes it, exactly as in the paper's form
// E = s^T A s + b^T s with A = cQ J, b = cH h:
//   1. determined: 2|cQ| S_i < |b_i|, S_i = sum of |J_ij| over alive
//      neighbours in row order (Eq. determined spin), s_i = -sgn(b_i);
//   2. each alive spin pulls b_j += sum over determined neighbours of
//      (2 cQ J_ji) s_i, summed in row order from 0 and added once;
//   3. isolated spins with b = 0 are fixed to +1 (optional extension);
//   4. semi-determined: one alive neighbour p and 2|cQ||J_kp| >= |b_k|
//      (Eq. semi determined spin); a mutual pair keeps only the larger index;
//      s_k = -sgn(cQ J_kp) s_p, the parent pulls b_p += sum of -sgn(cQ J_kp) b_k.
// All FP64 arithmetic uses explicit round-to-nearest intrinsics (no FMA
// contraction), so the decisions match a sequential FP64 evaluation bit for
// bit. Each fixed spin records its own share of the constant; the constant is
// their sum by a fixed-order reduction.
#include "common.cuh"

#include <algorithm>
#include <cmath>

namespace ising {
namespace {

enum : int8_t { KG = 0, KD = 1, KZ = 2, KS = 3 };

struct PruneDev {
  int64_t n;
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;  // stored couplings as double
  uint8_t* alive;
  uint8_t* isD;
  uint8_t* cand;
  uint8_t* isS;
  int8_t* kind;
  int32_t* rnd;
  int8_t* value;
  int32_t* parent;
  int8_t* psign;
  int32_t* par;   // single alive neighbour (this round)
  double* jkp;    // coupling to it
  double* b;      // paper-form field
  double* contrib;
  unsigned int* count;  // spins fixed this round
  unsigned int* nD;     // spins determined this round
  unsigned int* nS;     // spins semi-determined this round
  double cq, twocq, twocq_abs;
};

constexpr unsigned kFull = 0xffffffffu;

// Row kernels: one warp per row, lane l holding edge e0 + l of each chunk of
// 32 (coalesced loads). Sums whose decisions depend on their rounding are
// formed in row order: the relevant edges of a chunk are flagged by ballot
// and added one after another from lane 0 up, so every lane holds exactly
// the sequential sum.
__device__ __forceinline__ double add_in_order(double acc, double term, unsigned mask) {
  while (mask) {
    const int k = __ffs(mask) - 1;
    acc = __dadd_rn(acc, __shfl_sync(kFull, term, k));
    mask &= mask - 1;
  }
  return acc;
}

struct WarpRows {
  int lane;
  int64_t first, stride;
  __device__ WarpRows() {
    lane = threadIdx.x & 31;
    first = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  }
};

// Determined spins: 2|cQ| S_i < |b_i|. The lanes' partial sums, reduced by a
// butterfly (every lane gets the same value), give S in some order; any
// order of a sum of m nonnegative terms lies within gamma_(m-1) S of S, so
// the comparison is certain unless 2|cQ| S is within that bound of |b_i|,
// and only then is S summed again in row order.
__global__ void k_determined(PruneDev P) {
  const WarpRows w;
  for (int64_t i = w.first; i < P.n; i += w.stride) {
    uint8_t d = 0;
    if (P.alive[i]) {
      const int e0 = P.rowptr[i], e1 = P.rowptr[i + 1];
      double s = 0.0;
      for (int e = e0 + w.lane; e < e1; e += 32) {
        const double x = P.val[e];
        if (x != 0.0 && P.alive[P.col[e]]) s = __dadd_rn(s, fabs(x));
      }
      for (int o = 16; o; o >>= 1) s = __dadd_rn(s, __shfl_xor_sync(kFull, s, o));
      const double bi = fabs(P.b[i]);
      const double eps = (4.0 * (double)(e1 - e0) + 16.0) * 0x1p-53;
      const double ts = __dmul_rn(P.twocq_abs, s);
      if (__dmul_rn(ts, 1.0 - eps) > bi) {
        d = 0;
      } else if (__dmul_rn(ts, 1.0 + eps) < bi) {
        d = 1;
      } else {
        double S = 0.0;
        for (int c = e0; c < e1; c += 32) {
          const int e = c + w.lane;
          double term = 0.0;
          if (e < e1) {
            const double x = P.val[e];
            if (x != 0.0 && P.alive[P.col[e]]) term = fabs(x);
          }
          S = add_in_order(S, term, __ballot_sync(kFull, term != 0.0));
        }
        d = __dmul_rn(P.twocq_abs, S) < bi;
      }
    }
    if (w.lane == 0) {
      if (d) {
        P.value[i] = P.b[i] < 0.0 ? 1 : -1;
        atomicAdd(P.nD, 1u);
      }
      P.isD[i] = d;
    }
  }
}

__global__ void k_fold_determined(PruneDev P, int r) {
  if (*P.nD == 0) return;  // nothing determined this round
  const WarpRows w;
  for (int64_t i = w.first; i < P.n; i += w.stride) {
    if (!P.alive[i]) continue;
    const int e0 = P.rowptr[i], e1 = P.rowptr[i + 1];
    if (P.isD[i]) {
      // own share of the constant: b_i s_i + sum over determined neighbours of cQ J_ij s_i s_j
      const double si = (double)P.value[i];
      double c = __dmul_rn(P.b[i], si);
      for (int cb = e0; cb < e1; cb += 32) {
        const int e = cb + w.lane;
        double term = 0.0;
        bool rel = false;
        if (e < e1) {
          const int32_t j = P.col[e];
          const double x = P.val[e];
          if (x != 0.0 && P.isD[j]) {
            rel = true;
            term = __dmul_rn(__dmul_rn(__dmul_rn(P.cq, x), si), (double)P.value[j]);
          }
        }
        c = add_in_order(c, term, __ballot_sync(kFull, rel));
      }
      if (w.lane == 0) {
        P.contrib[i] = c;
        P.kind[i] = KD;
        P.rnd[i] = r;
        atomicAdd(P.count, 1u);
      }
    } else {
      double acc = 0.0;
      bool recv = false;
      for (int cb = e0; cb < e1; cb += 32) {
        const int e = cb + w.lane;
        double term = 0.0;
        bool rel = false;
        if (e < e1) {
          const int32_t j = P.col[e];
          const double x = P.val[e];
          if (x != 0.0 && P.isD[j]) {
            rel = true;
            term = __dmul_rn(__dmul_rn(P.twocq, x), (double)P.value[j]);
          }
        }
        const unsigned mask = __ballot_sync(kFull, rel);
        recv |= mask != 0u;
        acc = add_in_order(acc, term, mask);
      }
      if (recv && w.lane == 0) P.b[i] = __dadd_rn(P.b[i], acc);
    }
  }
}

// Alive, undetermined neighbours: their count, and the last of them in row
// order (the single neighbour when the count is one).
__global__ void k_degree(PruneDev P, int r, bool zero_rule) {
  const WarpRows w;
  for (int64_t i = w.first; i < P.n; i += w.stride) {
    uint8_t c = 0;
    if (P.alive[i] && !P.isD[i]) {
      const int e0 = P.rowptr[i], e1 = P.rowptr[i + 1];
      int deg = 0;
      int32_t p = -1;
      double jv = 0.0;
      for (int cb = e0; cb < e1; cb += 32) {
        const int e = cb + w.lane;
        int32_t j = 0;
        double x = 0.0;
        bool rel = false;
        if (e < e1) {
          j = P.col[e];
          x = P.val[e];
          rel = x != 0.0 && P.alive[j] && !P.isD[j];
        }
        const unsigned mask = __ballot_sync(kFull, rel);
        deg += __popc(mask);
        if (mask) {
          const int last = 31 - __clz(mask);
          p = __shfl_sync(kFull, j, last);
          jv = __shfl_sync(kFull, x, last);
        }
      }
      if (w.lane == 0) {
        if (deg == 0 && zero_rule && P.b[i] == 0.0) {
          P.kind[i] = KZ;
          P.rnd[i] = r;
          P.value[i] = 1;
          P.contrib[i] = 0.0;
          atomicAdd(P.count, 1u);
        } else if (deg == 1) {
          P.par[i] = p;
          P.jkp[i] = jv;
          c = __dmul_rn(P.twocq_abs, fabs(jv)) >= fabs(P.b[i]);
        }
      }
    }
    if (w.lane == 0) P.cand[i] = c;
  }
}

__global__ void k_remove_determined(PruneDev P) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (P.alive[i] && (P.isD[i] || P.kind[i] == KZ)) P.alive[i] = 0;
}

__global__ void k_select_semi(PruneDev P) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P.n;
       k += (int64_t)gridDim.x * blockDim.x) {
    uint8_t s = 0;
    if (P.cand[k]) {
      int32_t p = P.par[k];
      bool mutual = P.cand[p] && P.par[p] == (int32_t)k;
      s = !(mutual && (int32_t)k < p);
    }
    P.isS[k] = s;
    if (s) atomicAdd(P.nS, 1u);
  }
}

__global__ void k_fold_semi(PruneDev P, int r) {
  if (*P.nS == 0) return;  // no semi-determined spins this round
  const WarpRows w;
  for (int64_t i = w.first; i < P.n; i += w.stride) {
    if (!P.alive[i]) continue;
    if (P.isS[i]) {
      if (w.lane == 0) {
        const double jv = P.jkp[i];
        const double prod = __dmul_rn(P.cq, jv);
        P.psign[i] = prod > 0.0 ? -1 : 1;
        P.parent[i] = P.par[i];
        P.contrib[i] = -__dmul_rn(P.twocq_abs, fabs(jv));
        P.kind[i] = KS;
        P.rnd[i] = r;
        atomicAdd(P.count, 1u);
      }
    } else {
      const int e0 = P.rowptr[i], e1 = P.rowptr[i + 1];
      double acc = 0.0;
      bool recv = false;
      for (int cb = e0; cb < e1; cb += 32) {
        const int e = cb + w.lane;
        double term = 0.0;
        bool rel = false;
        if (e < e1) {
          const int32_t k = P.col[e];
          const double x = P.val[e];
          if (x != 0.0 && P.isS[k]) {
            rel = true;
            const double sg = __dmul_rn(P.cq, P.jkp[k]) > 0.0 ? -1.0 : 1.0;
            term = __dmul_rn(sg, P.b[k]);
          }
        }
        const unsigned mask = __ballot_sync(kFull, rel);
        recv |= mask != 0u;
        acc = add_in_order(acc, term, mask);
      }
      if (recv && w.lane == 0) P.b[i] = __dadd_rn(P.b[i], acc);
    }
  }
}

__global__ void k_remove_semi(PruneDev P) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (P.isS[i]) P.alive[i] = 0;
}

__global__ void k_init(PruneDev P, const void* h, int h_dtype, double ch) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    P.alive[i] = 1;
    P.kind[i] = KG;
    P.rnd[i] = 0;
    P.value[i] = 0;
    P.parent[i] = -1;
    P.psign[i] = 0;
    P.par[i] = -1;
    P.contrib[i] = 0.0;
    P.b[i] = h ? __dmul_rn(ch, load_as_double(h, h_dtype, i)) : 0.0;
  }
}

__global__ void k_values_double(const void* J, int dt, int64_t count, double* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = load_as_double(J, dt, e);
}

// Dense -> CSR (non-zero entries, increasing column), used by pruning only:
// a warp per row, 32 columns per ballot, positions from the ballot prefix.
__global__ void k_dense_count(const void* J, int dt, int64_t n, int32_t* cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    int c = 0;
    for (int64_t j0 = 0; j0 < n; j0 += 32) {
      const int64_t j = j0 + lane;
      c += __popc(__ballot_sync(0xffffffffu, j < n && load_as_double(J, dt, i * n + j) != 0.0));
    }
    if (lane == 0) cnt[i] = c;
  }
}

__global__ void k_dense_fill(const void* J, int dt, int64_t n, const int32_t* rowptr,
                             int32_t* col, double* val) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    int o = rowptr[i];
    for (int64_t j0 = 0; j0 < n; j0 += 32) {
      const int64_t j = j0 + lane;
      const double x = j < n ? load_as_double(J, dt, i * n + j) : 0.0;
      const unsigned int m = __ballot_sync(0xffffffffu, x != 0.0);
      if (x != 0.0) {
        const int pos = o + __popc(m & ((1u << lane) - 1u));
        col[pos] = (int32_t)j;
        val[pos] = x;
      }
      o += __popc(m);
    }
  }
}

// Reduced CSR: kept entries of kept rows, columns relabelled (order kept).
__global__ void k_reduced_count(PruneDev P, const int64_t* G, int64_t nG, int32_t* cnt) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nG;
       g += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = G[g];
    int c = 0;
    for (int e = P.rowptr[i]; e < P.rowptr[i + 1]; ++e)
      c += P.val[e] != 0.0 && P.alive[P.col[e]];
    cnt[g] = c;
  }
}

__global__ void k_reduced_fill(PruneDev P, const int64_t* G, int64_t nG, const int64_t* gidx,
                               const int64_t* rp, const void* Jsrc, int dt, size_t esz,
                               int32_t* cols, void* vals) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nG;
       g += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = G[g];
    int64_t o = rp[g];
    for (int e = P.rowptr[i]; e < P.rowptr[i + 1]; ++e) {
      int32_t j = P.col[e];
      if (P.val[e] != 0.0 && P.alive[j]) {
        cols[o] = (int32_t)gidx[j];
        memcpy(static_cast<char*>(vals) + o * esz, static_cast<const char*>(Jsrc) + (int64_t)e * esz, esz);
        ++o;
      }
    }
  }
}

__global__ void k_reduced_dense(const void* J, size_t esz, int64_t n, const int64_t* G,
                                int64_t nG, void* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nG * nG;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t a = e / nG, c = e - a * nG;
    memcpy(static_cast<char*>(out) + e * esz,
           static_cast<const char*>(J) + (G[a] * n + G[c]) * esz, esz);
  }
}

__global__ void k_reduced_h(const double* b, double ch, const int64_t* G, int64_t nG, double* h) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nG;
       g += (int64_t)gridDim.x * blockDim.x)
    h[g] = __dmul_rn(ch, b[G[g]]);
}

// Fixed-order sum of the per-spin shares of the constant (one block).
__global__ void __launch_bounds__(1024) k_sum(const double* x, int64_t n, double* out) {
  __shared__ double sh[1024];
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a = __dadd_rn(a, x[i]);
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = __dadd_rn(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// K5: s_i for every original spin: kept spins copy the reduced solution,
// fixed spins their value, semi-determined spins follow the parent chain.
__global__ void k_reconstruct(int64_t n, const int8_t* kind, const int8_t* value,
                              const int32_t* parent, const int8_t* psign, const int64_t* gidx,
                              const int8_t* sG, int8_t* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int sign = 1;
    int64_t p = i;
    for (int64_t hops = 0; kind[p] == KS && hops < n; ++hops) {
      sign *= psign[p];
      p = parent[p];
    }
    int8_t base = kind[p] == KG ? sG[gidx[p]] : value[p];
    out[i] = (int8_t)(sign * base);
  }
}

int grid_n(ising_ctx* ctx, int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)ctx->sm_count * 8));
}

}  // namespace
}  // namespace ising

using namespace ising;

struct ising_prune_result {
  ising_ctx* ctx = nullptr;
  int64_t n = 0, nG = 0, nnzG = 0;
  int layout = ISING_LAYOUT_CSR;
  int j_dtype = ISING_F64;
  double j_scale = 1.0;
  int convention = ISING_CONV_PHYSICS;
  double constant = 0.0, eta = 0.0;
  int rounds = 0;
  DevMem kind, rnd, value, parent, psign, gidx;
  DevMem Jr, indptr_r, indices_r, h_r;
};

namespace ising {
int prune_device(ising_ctx* ctx, const DevInstance& I, int flags, ising_prune_result** out);
}

extern "C" int ising_prune(ising_ctx* ctx, const ising_instance* inst, int flags,
                           ising_prune_result** out) {
  if (!ctx) return ISING_EINVAL;
  if (!out) return fail(ctx, ISING_EINVAL, "out is NULL");
  if (flags & ~ISING_PRUNE_ZERO_RULE) return fail(ctx, ISING_EINVAL, "unknown prune flags");
  *out = nullptr;
  ISING_CUDA(ctx, cudaSetDevice(ctx->device));
  DevInstance I;
  ISING_TRY(upload_instance(ctx, inst, &I));
  return ising::prune_device(ctx, I, flags, out);
}

// Algorithm 1 on an uploaded, validated instance.
int ising::prune_device(ising_ctx* ctx, const DevInstance& I, int flags,
                        ising_prune_result** out) {
  *out = nullptr;
  cudaStream_t st = ctx->stream;
  const int64_t n = I.n;
  // CSR view with double values
  DevMem rowptr, col, val;
  int64_t nnz;
  if (I.layout == ISING_LAYOUT_CSR) {
    nnz = I.nnz;
    ISING_TRY(dev_alloc(ctx, val, nnz * 8));
    if (nnz) k_values_double<<<grid_n(ctx, nnz), 256, 0, st>>>(I.J.p, I.j_dtype, nnz, val.as<double>());
  } else {
    DevMem cnt;
    ISING_TRY(dev_alloc(ctx, cnt, n * 4));
    k_dense_count<<<grid_n(ctx, n * 32), 256, 0, st>>>(I.J.p, I.j_dtype, n, cnt.as<int32_t>());
    std::vector<int32_t> c(n), rp(n + 1);
    ISING_CUDA(ctx, cudaMemcpyAsync(c.data(), cnt.p, n * 4, cudaMemcpyDeviceToHost, st));
    ISING_CUDA(ctx, cudaStreamSynchronize(st));
    rp[0] = 0;
    for (int64_t i = 0; i < n; ++i) rp[i + 1] = rp[i] + c[i];
    nnz = rp[n];
    ISING_TRY(dev_alloc(ctx, rowptr, (n + 1) * 4));
    ISING_TRY(dev_alloc(ctx, col, nnz * 4));
    ISING_TRY(dev_alloc(ctx, val, nnz * 8));
    ISING_CUDA(ctx, cudaMemcpyAsync(rowptr.p, rp.data(), (n + 1) * 4, cudaMemcpyHostToDevice, st));
    k_dense_fill<<<grid_n(ctx, n * 32), 256, 0, st>>>(I.J.p, I.j_dtype, n, rowptr.as<int32_t>(),
                                                 col.as<int32_t>(), val.as<double>());
    ISING_CUDA(ctx, cudaStreamSynchronize(st));
  }
  ISING_CUDA(ctx, cudaGetLastError());
  auto res = new ising_prune_result();
  res->ctx = ctx;
  res->n = n;
  res->layout = I.layout;
  res->j_dtype = I.j_dtype;
  res->j_scale = I.j_scale;
  res->convention = I.convention;
  int rc = [&]() -> int {
    DevMem alive, isD, cand, isS, par, jkp, b, contrib, count;
    ISING_TRY(dev_alloc(ctx, alive, n));
    ISING_TRY(dev_alloc(ctx, isD, n));
    ISING_TRY(dev_alloc(ctx, cand, n));
    ISING_TRY(dev_alloc(ctx, isS, n));
    ISING_TRY(dev_alloc(ctx, par, n * 4));
    ISING_TRY(dev_alloc(ctx, jkp, n * 8));
    ISING_TRY(dev_alloc(ctx, b, n * 8));
    ISING_TRY(dev_alloc(ctx, contrib, n * 8));
    ISING_TRY(dev_alloc(ctx, count, 16));
    ISING_TRY(dev_alloc(ctx, res->kind, n));
    ISING_TRY(dev_alloc(ctx, res->rnd, n * 4));
    ISING_TRY(dev_alloc(ctx, res->value, n));
    ISING_TRY(dev_alloc(ctx, res->parent, n * 4));
    ISING_TRY(dev_alloc(ctx, res->psign, n));
    ISING_TRY(dev_alloc(ctx, res->gidx, n * 8));
    PruneDev P;
    P.n = n;
    P.rowptr = I.layout == ISING_LAYOUT_CSR ? I.rowptr.as<int32_t>() : rowptr.as<int32_t>();
    P.col = I.layout == ISING_LAYOUT_CSR ? I.indices.as<int32_t>() : col.as<int32_t>();
    P.val = val.as<double>();
    P.alive = alive.as<uint8_t>();
    P.isD = isD.as<uint8_t>();
    P.cand = cand.as<uint8_t>();
    P.isS = isS.as<uint8_t>();
    P.kind = res->kind.as<int8_t>();
    P.rnd = res->rnd.as<int32_t>();
    P.value = res->value.as<int8_t>();
    P.parent = res->parent.as<int32_t>();
    P.psign = res->psign.as<int8_t>();
    P.par = par.as<int32_t>();
    P.jkp = jkp.as<double>();
    P.b = b.as<double>();
    P.contrib = contrib.as<double>();
    P.count = count.as<unsigned int>();
    P.nD = count.as<unsigned int>() + 1;
    P.nS = count.as<unsigned int>() + 2;
    P.cq = I.cq;
    P.twocq = 2.0 * I.cq;
    P.twocq_abs = std::fabs(2.0 * I.cq);
    const int g = grid_n(ctx, n);
    const int gw = grid_n(ctx, n * 32);  // warp-per-row kernels
    k_init<<<g, 256, 0, st>>>(P, I.has_h ? I.h.p : nullptr, I.h_dtype, I.ch);
    ISING_CUDA(ctx, cudaGetLastError());
    const bool zero_rule = (flags & ISING_PRUNE_ZERO_RULE) != 0;
    int rounds = 0;
    for (int r = 1; r <= n + 1; ++r) {
      ISING_CUDA(ctx, cudaMemsetAsync(count.p, 0, 12, st));
      k_determined<<<gw, 256, 0, st>>>(P);
      k_fold_determined<<<gw, 256, 0, st>>>(P, r);
      k_degree<<<gw, 256, 0, st>>>(P, r, zero_rule);
      k_remove_determined<<<g, 256, 0, st>>>(P);
      k_select_semi<<<g, 256, 0, st>>>(P);
      k_fold_semi<<<gw, 256, 0, st>>>(P, r);
      k_remove_semi<<<g, 256, 0, st>>>(P);
      ISING_CUDA(ctx, cudaGetLastError());
      unsigned int changed = 0;
      ISING_CUDA(ctx, cudaMemcpyAsync(&changed, count.p, 4, cudaMemcpyDeviceToHost, st));
      ISING_CUDA(ctx, cudaStreamSynchronize(st));
      if (!changed) break;
      rounds = r;
    }
    res->rounds = rounds;
    // kept spins, increasing original index
    std::vector<uint8_t> al(n);
    ISING_CUDA(ctx, cudaMemcpyAsync(al.data(), alive.p, n, cudaMemcpyDeviceToHost, st));
    ISING_CUDA(ctx, cudaStreamSynchronize(st));
    std::vector<int64_t> G, gi(n, -1);
    for (int64_t i = 0; i < n; ++i)
      if (al[i]) { gi[i] = (int64_t)G.size(); G.push_back(i); }
    const int64_t nG = (int64_t)G.size();
    res->nG = nG;
    res->eta = 1.0 - (double)nG / (double)n;
    ISING_CUDA(ctx, cudaMemcpyAsync(res->gidx.p, gi.data(), n * 8, cudaMemcpyHostToDevice, st));
    DevMem Gd, csum;
    ISING_TRY(dev_alloc(ctx, Gd, std::max<int64_t>(nG, 1) * 8));
    ISING_TRY(dev_alloc(ctx, csum, 8));
    if (nG) ISING_CUDA(ctx, cudaMemcpyAsync(Gd.p, G.data(), nG * 8, cudaMemcpyHostToDevice, st));
    k_sum<<<1, 1024, 0, st>>>(contrib.as<double>(), n, csum.as<double>());
    ISING_CUDA(ctx, cudaMemcpyAsync(&res->constant, csum.p, 8, cudaMemcpyDeviceToHost, st));
    const size_t esz = dtype_size(I.j_dtype);
    ISING_TRY(dev_alloc(ctx, res->h_r, std::max<int64_t>(nG, 1) * 8));
    if (nG) k_reduced_h<<<grid_n(ctx, nG), 256, 0, st>>>(P.b, I.ch, Gd.as<int64_t>(), nG, res->h_r.as<double>());
    if (I.layout == ISING_LAYOUT_DENSE) {
      ISING_TRY(dev_alloc(ctx, res->Jr, std::max<int64_t>(nG * nG, 1) * esz));
      if (nG)
        k_reduced_dense<<<grid_n(ctx, nG * nG), 256, 0, st>>>(I.J.p, esz, n, Gd.as<int64_t>(),
                                                              nG, res->Jr.p);
      res->nnzG = nG * nG;
    } else {
      DevMem cnt;
      ISING_TRY(dev_alloc(ctx, cnt, std::max<int64_t>(nG, 1) * 4));
      std::vector<int32_t> c(nG);
      if (nG) {
        k_reduced_count<<<grid_n(ctx, nG), 256, 0, st>>>(P, Gd.as<int64_t>(), nG, cnt.as<int32_t>());
        ISING_CUDA(ctx, cudaMemcpyAsync(c.data(), cnt.p, nG * 4, cudaMemcpyDeviceToHost, st));
        ISING_CUDA(ctx, cudaStreamSynchronize(st));
      }
      std::vector<int64_t> rp(nG + 1, 0);
      for (int64_t a = 0; a < nG; ++a) rp[a + 1] = rp[a] + c[a];
      res->nnzG = rp[nG];
      ISING_TRY(dev_alloc(ctx, res->indptr_r, (nG + 1) * 8));
      ISING_TRY(dev_alloc(ctx, res->indices_r, std::max<int64_t>(res->nnzG, 1) * 4));
      ISING_TRY(dev_alloc(ctx, res->Jr, std::max<int64_t>(res->nnzG, 1) * esz));
      ISING_CUDA(ctx, cudaMemcpyAsync(res->indptr_r.p, rp.data(), (nG + 1) * 8, cudaMemcpyHostToDevice, st));
      if (nG)
        k_reduced_fill<<<grid_n(ctx, nG), 256, 0, st>>>(P, Gd.as<int64_t>(), nG, res->gidx.as<int64_t>(),
                                                        res->indptr_r.as<int64_t>(), I.J.p, I.j_dtype,
                                                        esz, res->indices_r.as<int32_t>(), res->Jr.p);
    }
    ISING_CUDA(ctx, cudaGetLastError());
    ISING_CUDA(ctx, cudaStreamSynchronize(st));
    return ISING_OK;
  }();
  if (rc != ISING_OK) {
    delete res;
    return rc;
  }
  *out = res;
  return ISING_OK;
}

extern "C" int ising_prune_info(const ising_prune_result* res, int64_t* n_reduced,
                                int64_t* nnz_reduced, double* constant, double* eta,
                                int32_t* rounds) {
  if (!res) return ISING_EINVAL;
  if (n_reduced) *n_reduced = res->nG;
  if (nnz_reduced) *nnz_reduced = res->nnzG;
  if (constant) *constant = res->constant;
  if (eta) *eta = res->eta;
  if (rounds) *rounds = res->rounds;
  return ISING_OK;
}

extern "C" int ising_prune_reduced(const ising_prune_result* res, ising_instance* out) {
  if (!res || !out) return ISING_EINVAL;
  memset(out, 0, sizeof *out);
  out->n = res->nG;
  out->layout = res->layout;
  out->j_dtype = res->j_dtype;
  out->J = res->Jr.p;
  out->indptr = res->layout == ISING_LAYOUT_CSR ? res->indptr_r.as<int64_t>() : nullptr;
  out->indices = res->layout == ISING_LAYOUT_CSR ? res->indices_r.as<int32_t>() : nullptr;
  out->nnz = res->nnzG;
  out->h_dtype = ISING_F64;
  out->h = res->h_r.p;
  out->j_scale = res->j_scale;
  out->convention = res->convention;
  out->mem = ISING_MEM_DEVICE;
  return ISING_OK;
}

extern "C" int ising_prune_reduced_copy(const ising_prune_result* res, void* J, int64_t* indptr,
                                        int32_t* indices, double* h, int mem) {
  if (!res) return ISING_EINVAL;
  ising_ctx* ctx = res->ctx;
  if (mem != ISING_MEM_HOST && mem != ISING_MEM_DEVICE) return fail(ctx, ISING_EINVAL, "bad mem");
  cudaMemcpyKind k = mem == ISING_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const size_t esz = dtype_size(res->j_dtype);
  if (J && res->nnzG) ISING_CUDA(ctx, cudaMemcpyAsync(J, res->Jr.p, res->nnzG * esz, k, ctx->stream));
  if (res->layout == ISING_LAYOUT_CSR) {
    if (indptr) ISING_CUDA(ctx, cudaMemcpyAsync(indptr, res->indptr_r.p, (res->nG + 1) * 8, k, ctx->stream));
    if (indices && res->nnzG)
      ISING_CUDA(ctx, cudaMemcpyAsync(indices, res->indices_r.p, res->nnzG * 4, k, ctx->stream));
  }
  if (h && res->nG) ISING_CUDA(ctx, cudaMemcpyAsync(h, res->h_r.p, res->nG * 8, k, ctx->stream));
  ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ISING_OK;
}

extern "C" int ising_prune_record(const ising_prune_result* res, int8_t* kind, int32_t* round,
                                  int8_t* value, int32_t* parent, int8_t* sign,
                                  int64_t* g_index, int mem) {
  if (!res) return ISING_EINVAL;
  ising_ctx* ctx = res->ctx;
  if (mem != ISING_MEM_HOST && mem != ISING_MEM_DEVICE) return fail(ctx, ISING_EINVAL, "bad mem");
  cudaMemcpyKind k = mem == ISING_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const int64_t n = res->n;
  if (kind) ISING_CUDA(ctx, cudaMemcpyAsync(kind, res->kind.p, n, k, ctx->stream));
  if (round) ISING_CUDA(ctx, cudaMemcpyAsync(round, res->rnd.p, n * 4, k, ctx->stream));
  if (value) ISING_CUDA(ctx, cudaMemcpyAsync(value, res->value.p, n, k, ctx->stream));
  if (parent) ISING_CUDA(ctx, cudaMemcpyAsync(parent, res->parent.p, n * 4, k, ctx->stream));
  if (sign) ISING_CUDA(ctx, cudaMemcpyAsync(sign, res->psign.p, n, k, ctx->stream));
  if (g_index) ISING_CUDA(ctx, cudaMemcpyAsync(g_index, res->gidx.p, n * 8, k, ctx->stream));
  ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ISING_OK;
}

extern "C" int ising_prune_free(ising_prune_result* res) {
  if (res && res->ctx) cudaStreamSynchronize(res->ctx->stream);
  delete res;
  return ISING_OK;
}

extern "C" int ising_reconstruct(ising_ctx* ctx, const ising_prune_result* res,
                                 const int8_t* reduced_spins, int8_t* full_spins, int mem) {
  if (!ctx || !res) return ISING_EINVAL;
  if (!full_spins || (!reduced_spins && res->nG > 0))
    return fail(ctx, ISING_EINVAL, "spin buffers are NULL");
  if (mem != ISING_MEM_HOST && mem != ISING_MEM_DEVICE) return fail(ctx, ISING_EINVAL, "bad mem");
  cudaStream_t st = ctx->stream;
  DevMem sG, out;
  const int8_t* sg = reduced_spins;
  int8_t* o = full_spins;
  if (mem == ISING_MEM_HOST) {
    ISING_TRY(dev_alloc(ctx, sG, std::max<int64_t>(res->nG, 1)));
    ISING_TRY(dev_alloc(ctx, out, res->n));
    if (res->nG) ISING_CUDA(ctx, cudaMemcpyAsync(sG.p, reduced_spins, res->nG, cudaMemcpyHostToDevice, st));
    sg = sG.as<int8_t>();
    o = out.as<int8_t>();
  }
  k_reconstruct<<<grid_n(ctx, res->n), 256, 0, st>>>(
      res->n, res->kind.as<int8_t>(), res->value.as<int8_t>(), res->parent.as<int32_t>(),
      res->psign.as<int8_t>(), res->gidx.as<int64_t>(), sg, o);
  ISING_CUDA(ctx, cudaGetLastError());
  if (mem == ISING_MEM_HOST)
    ISING_CUDA(ctx, cudaMemcpyAsync(full_spins, out.p, res->n, cudaMemcpyDeviceToHost, st));
  ISING_CUDA(ctx, cudaStreamSynchronize(st));
  return ISING_OK;
}
