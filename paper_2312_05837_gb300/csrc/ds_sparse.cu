// K2s: fused domain-selection step (Sec. III-B) for CSR couplings.
//
// Layout: state theta, m, v is [n][Bp] (restarts contiguous, Bp a multiple of
// 128); spins are bit-packed [n][Bp/32] words (bit set = +1). A block covers
// a range of rows and one 128-restart slice (grid.y); a warp owns one row at a
// time and lane l owns restarts 4 l + {0..3} of the slice, so every state
// access is a coalesced float4 and a neighbour's spins are one broadcast word
// per group of 8 lanes. A row's edges are read either by every lane
// (many rows per warp, the next row's state in flight meanwhile) or one edge
// per lane and broadcast (few rows per warp: the gathers then overlap); both
// visit the edges in order, so G is the same. The per-row epilogue is the
// same as the dense paths: F = cQ G + cH h - mu s, g = cos(theta) F, Adam,
// projection, new spin bit; energy partials of the input spins are summed
// per block in warp order. In the
// relaxed mode each neighbour also contributes J_ij x_j with x = sin(theta)
// from the FP32 slot x_t ([n][Bp], float4 per lane): that product drives the
// update, the bit product the energies, and x_{t+1} is written out.
#include "ds_internal.cuh"

#include <algorithm>

namespace ising {
namespace {

// Q = restarts per warp pass / 128. Q = 1 fits 64 registers (four blocks
// per SM); Q = 2 gathers each neighbour's spins once for 256 restarts (two
// blocks per SM). Both visit rows, lanes and partials in the same order,
// so their results are identical bit for bit.
// LANE: the few-rows-per-warp edge visit (small instances, whose grids are
// small too: two blocks per SM leave it the registers it needs).
template <int Q, int MODE, bool INT_E, bool VAL_I8, bool LANE>
__global__ void __launch_bounds__(256, LANE ? 2 : (Q == 1 ? (MODE == kModeRelaxed ? 3 : 4) : 2))
    sparse_step_kernel(
    int64_t n, int64_t Bp, int64_t rows_per_block, const int32_t* __restrict__ rowptr,
    const int32_t* __restrict__ col, const void* __restrict__ val,
    const uint32_t* __restrict__ bits_in, uint32_t* __restrict__ bits_out,
    float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
    const float* __restrict__ hf, const int32_t* __restrict__ hint, StepConsts k,
    const float2* __restrict__ bias, const long long* __restrict__ counters,
    long long* __restrict__ qpart, long long* __restrict__ hpart, float* __restrict__ epart,
    float* __restrict__ Gout, const float* __restrict__ xin, float* __restrict__ xout,
    int64_t B, const int* __restrict__ live32, unsigned long long* __restrict__ work) {
  constexpr bool RELAXED = MODE == kModeRelaxed;
  constexpr bool UPDATE = MODE == kModeUpdate || RELAXED;
  constexpr int W = 8;  // warps per block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t words = Bp / 32;
  const int64_t cb = (int64_t)blockIdx.y * (128 * Q);  // first restart of this slice
  const int64_t ce = cb + 128 * Q < B ? cb + 128 * Q : B;
  if (MODE != kModeCoupling && restarts_retired(live32, cb, ce)) return;  // (uniform per block)
  if (UPDATE && work && blockIdx.x == 0 && threadIdx.x == 0)
    atomicAdd(work, (unsigned long long)(ce - cb));
  const int64_t wofs = cb / 32 + (lane >> 3);
  const int nshift = 4 * (lane & 7);
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < n ? r0 + rows_per_block : n;
  const float2 bc = bias[counters[0] + 1];

  int eq[Q][4], eh[Q][4];
  float ee[Q][4];
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int r = 0; r < 4; ++r) { eq[q][r] = 0; eh[q][r] = 0; ee[q][r] = 0.f; }

  // rows of this warp: r0 + warp, r0 + warp + W, ...; the state of the next
  // row is requested before the current row's neighbour gather (streamed once
  // per step, evict-first), so HBM latency overlaps the dependent gather
  float4 th_n[Q], m_n[Q], v_n[Q];
  uint32_t own_n[Q];
  int rb_n = 0, re_n = 0;
  auto fetch = [&](int64_t row) {
    rb_n = rowptr[row];
    re_n = rowptr[row + 1];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int64_t base = row * Bp + cb + 128 * q + 4 * lane;
      if (UPDATE) {
        th_n[q] = __ldcs(reinterpret_cast<const float4*>(theta + base));
        m_n[q] = __ldcs(reinterpret_cast<const float4*>(m + base));
        v_n[q] = __ldcs(reinterpret_cast<const float4*>(v + base));
      }
      own_n[q] = (bits_in[row * words + wofs + 4 * q] >> nshift) & 0xFu;
    }
  };
  if (r0 + warp < r1) fetch(r0 + warp);
  for (int64_t i = r0 + warp; i < r1; i += W) {
    float4 th4[Q], m4[Q], v4[Q];
    uint32_t own[Q];
    const int rb = rb_n, re = re_n;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      th4[q] = th_n[q];
      m4[q] = m_n[q];
      v4[q] = v_n[q];
      own[q] = own_n[q];
    }
    if (i + W < r1) fetch(i + W);
    float G[Q][4], Gx[Q][4];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) { G[q][r] = 0.f; Gx[q][r] = 0.f; }
    auto add_edge = [&](int64_t j, float Jv, const uint32_t* w) {
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const uint32_t nib = (w[q] >> nshift) & 0xFu;
#pragma unroll
        for (int r = 0; r < 4; ++r) G[q][r] += ((nib >> r) & 1u) ? Jv : -Jv;
        if (RELAXED) {
          const float4 xj = __ldg(reinterpret_cast<const float4*>(xin + j * Bp + cb + 128 * q + 4 * lane));
          Gx[q][0] = fmaf(Jv, xj.x, Gx[q][0]);
          Gx[q][1] = fmaf(Jv, xj.y, Gx[q][1]);
          Gx[q][2] = fmaf(Jv, xj.z, Gx[q][2]);
          Gx[q][3] = fmaf(Jv, xj.w, Gx[q][3]);
        }
      }
    };
    if constexpr (LANE) {
      // few rows per warp (small instances): the row's edges, up to 32 at a
      // time, lane k loading edge k (one coalesced load); then the spin
      // words of several edges at once, lane L loading word L % (4 Q) of
      // edge L / (4 Q) (a row's words for this slice are contiguous), so one
      // load instruction covers 32 / (4 Q) edges; the edges are then added
      // in order, each lane taking its words by shuffle
      constexpr int kWpe = 4 * Q;       // words per edge in this slice
      constexpr int kEpp = 32 / kWpe;   // edges per load pass
      for (int eb = rb; eb < re; eb += 32) {
        const int cnt = re - eb < 32 ? re - eb : 32;
        int jl = 0;
        float vl = 0.f;
        if (lane < cnt) {
          jl = col[eb + lane];
          vl = VAL_I8 ? (float)static_cast<const int8_t*>(val)[eb + lane]
                      : static_cast<const float*>(val)[eb + lane];
        }
#pragma unroll 1
        for (int p0 = 0; p0 < cnt; p0 += kEpp) {
          const int ke = p0 + lane / kWpe;  // < 32
          const int64_t jk = __shfl_sync(0xffffffffu, jl, ke);
          uint32_t wv = 0u;
          if (ke < cnt) wv = __ldg(&bits_in[jk * words + cb / 32 + lane % kWpe]);
          const int ne = cnt - p0 < kEpp ? cnt - p0 : kEpp;
#pragma unroll 1
          for (int e = 0; e < ne; ++e) {
            const int64_t j = __shfl_sync(0xffffffffu, jl, p0 + e);
            const float Jv = __shfl_sync(0xffffffffu, vl, p0 + e);
            uint32_t w[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q)
              w[q] = __shfl_sync(0xffffffffu, wv, e * kWpe + 4 * q + (lane >> 3));
            add_edge(j, Jv, w);
          }
        }
      }
    } else {
      // many rows per warp: every lane reads each edge (broadcast) and the
      // next row's state is already in flight
#pragma unroll (RELAXED ? 1 : 4)
      for (int e = rb; e < re; ++e) {
        const int64_t j = col[e];
        const float Jv = VAL_I8 ? (float)static_cast<const int8_t*>(val)[e]
                                : static_cast<const float*>(val)[e];
        uint32_t w[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) w[q] = __ldg(&bits_in[j * words + wofs + 4 * q]);
        add_edge(j, Jv, w);
      }
    }
    if (MODE == kModeCoupling) {
#pragma unroll
      for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) Gout[i * Bp + cb + 128 * q + 4 * lane + r] = G[q][r];
      continue;
    }
    const float h = hf[i];
    const int hi = hint[i];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int64_t base = i * Bp + cb + 128 * q + 4 * lane;
      float* thp = &th4[q].x;
      float* mp = &m4[q].x;
      float* vp = &v4[q].x;
      uint32_t newnib = 0;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float s = ((own[q] >> r) & 1u) ? 1.f : -1.f;
        if (INT_E) {
          eq[q][r] += (int)s * __float2int_rn(G[q][r]);
          eh[q][r] += (int)s * hi;
        } else {
          ee[q][r] += s * fmaf(k.cq, G[q][r], k.ch * h);
        }
        if (UPDATE) {
          const float F = fmaf(k.cq, RELAXED ? Gx[q][r] : G[q][r], fmaf(k.ch, h, -k.mu * s));
          const float g = cos_proj(thp[r]) * F;
          thp[r] = adam_update(k, bc.x, bc.y, g, thp[r], mp[r], vp[r]);
          if (sin_nonneg(thp[r])) newnib |= 1u << r;
        }
      }
      if (UPDATE) {
        __stcs(reinterpret_cast<float4*>(theta + base), th4[q]);
        __stcs(reinterpret_cast<float4*>(m + base), m4[q]);
        __stcs(reinterpret_cast<float4*>(v + base), v4[q]);
        if (RELAXED)
          *reinterpret_cast<float4*>(xout + base) =
              make_float4(sin_proj(th4[q].x), sin_proj(th4[q].y), sin_proj(th4[q].z), sin_proj(th4[q].w));
        uint32_t word = newnib << nshift;
        word |= __shfl_xor_sync(0xffffffffu, word, 1);
        word |= __shfl_xor_sync(0xffffffffu, word, 2);
        word |= __shfl_xor_sync(0xffffffffu, word, 4);
        if ((lane & 7) == 0) bits_out[i * words + wofs + 4 * q] = word;
      }
    }
  }

  // energy partials: per restart, sum over this block's rows in warp order
  if (MODE == kModeCoupling) return;
  __shared__ float red_f[INT_E ? 1 : W][INT_E ? 1 : 128 * Q];
  __shared__ int red_q[INT_E ? W : 1][INT_E ? 128 * Q : 1];
  __shared__ int red_h[INT_E ? W : 1][INT_E ? 128 * Q : 1];
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int c = 128 * q + 4 * lane + r;
      if (INT_E) {
        red_q[warp][c] = eq[q][r];
        red_h[warp][c] = eh[q][r];
      } else {
        red_f[warp][c] = ee[q][r];
      }
    }
  __syncthreads();
  for (int c = threadIdx.x; c < 128 * Q; c += blockDim.x) {
    const int64_t o = (int64_t)blockIdx.x * Bp + cb + c;
    if (INT_E) {
      long long a = 0, b = 0;
#pragma unroll
      for (int w = 0; w < W; ++w) { a += red_q[w][c]; b += red_h[w][c]; }
      qpart[o] = a;
      hpart[o] = b;
    } else {
      float a = 0.f;
#pragma unroll
      for (int w = 0; w < W; ++w) a += red_f[w][c];
      epart[o] = a;
    }
  }
}

__global__ void csr_values_kernel(const void* J, int dt, int64_t nnz, bool to_i8, void* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    double x = load_as_double(J, dt, e);
    if (to_i8) static_cast<int8_t*>(out)[e] = (int8_t)x;
    else static_cast<float*>(out)[e] = (float)x;
  }
}

// Row blocks: one wave of the Q = 1 kernel (four blocks per SM over the
// 128-restart slices), at least 8 rows (one per warp) each; a warp then
// streams its rows back to back with the next row's state in flight. Small
// instances thus spread over as many warps as they have rows.
int64_t sparse_rows_per_block(ising_ds* ds) {
  const int64_t slices = std::max<int64_t>(ds->Bp / 128, 1);
  const int64_t target = std::max<int64_t>((int64_t)ds->ctx->sm_count * 4 / slices, 1);
  const int64_t nb = std::min<int64_t>((ds->n + 7) / 8, target);
  return (ds->n + nb - 1) / nb;
}

}  // namespace

int sparse_setup(ising_ds* ds) {
  ising_ctx* ctx = ds->ctx;
  ds->Bp = (ds->B + 127) / 128 * 128;
  ds->ld = ds->n;
  ds->spin_kind = kSpinBits;
  const int64_t rpb = sparse_rows_per_block(ds);
  ds->mtiles = (int)((ds->n + rpb - 1) / rpb);
  ds->sp_int8 = ds->inst.j_integer && ds->inst.j_absmax <= 127.0;
  const int64_t nnz = ds->inst.nnz;
  ISING_TRY(dev_alloc(ctx, ds->sp_val, (size_t)nnz * (ds->sp_int8 ? 1 : 4)));
  if (nnz) {
    int g = (int)std::min<int64_t>((nnz + 255) / 256, (int64_t)ctx->sm_count * 16);
    csr_values_kernel<<<g, 256, 0, ctx->stream>>>(ds->inst.J.p, ds->inst.j_dtype, nnz,
                                                  ds->sp_int8, ds->sp_val.p);
    ISING_CUDA(ctx, cudaGetLastError());
  }
  return ISING_OK;
}

int sparse_step(ising_ds* ds, int mode, float* Gout) {
  ising_ctx* ctx = ds->ctx;
  const int64_t t = ds->t + 1;
  const uint32_t* in = ds->spins[t % 3].as<uint32_t>();
  uint32_t* out = ds->spins[(t + 1) % 3].as<uint32_t>();
  const int ps = (int)(t % 2);
  const int64_t rpb = sparse_rows_per_block(ds);
  const int Q = (ds->sp_q == 2 && (ds->Bp / 128) % 2 == 0) ? 2 : 1;
  const float* xin = mode == kModeRelaxed ? ds->xbuf[t % 2].as<float>() : nullptr;
  float* xout = mode == kModeRelaxed ? ds->xbuf[(t + 1) % 2].as<float>() : nullptr;
  dim3 grid((unsigned)ds->mtiles, (unsigned)(ds->Bp / (128 * Q)));
  const bool lane_edges = (rpb + 7) / 8 <= 4;  // rows per warp
#define ISING_SP(U, I, V)                                                                     \
  do {                                                                                        \
    if (Q == 2 && lane_edges)                                                                 \
      sparse_step_kernel<2, U, I, V, true><<<grid, 256, 0, ctx->stream>>>(ISING_SP_ARGS);     \
    else if (Q == 2)                                                                          \
      sparse_step_kernel<2, U, I, V, false><<<grid, 256, 0, ctx->stream>>>(ISING_SP_ARGS);    \
    else if (lane_edges)                                                                      \
      sparse_step_kernel<1, U, I, V, true><<<grid, 256, 0, ctx->stream>>>(ISING_SP_ARGS);     \
    else                                                                                      \
      sparse_step_kernel<1, U, I, V, false><<<grid, 256, 0, ctx->stream>>>(ISING_SP_ARGS);    \
  } while (0)
#define ISING_SP_ARGS                                                                         \
      ds->n, ds->Bp, rpb, ds->inst.rowptr.as<int32_t>(), ds->inst.indices.as<int32_t>(),      \
      ds->sp_val.p, in, out, ds->theta.as<float>(), ds->m.as<float>(), ds->v.as<float>(),     \
      ds->hf.as<float>(), ds->hint.as<int32_t>(), ds->k, ds->bias.as<float2>(),               \
      ds->counters.as<long long>(), ds->qpart[ps].as<long long>(),                            \
      ds->hpart[ps].as<long long>(), ds->epart[ps].as<float>(), Gout, xin, xout, ds->B,          \
      ds->live.p ? ds->live.as<int>() : nullptr, ds->work.as<unsigned long long>()
#define ISING_SP_V(U, I) \
  do { if (ds->sp_int8) ISING_SP(U, I, true); else ISING_SP(U, I, false); } while (0)
#define ISING_SP_I(U) \
  do { if (ds->int_energy) ISING_SP_V(U, true); else ISING_SP_V(U, false); } while (0)
  if (mode == kModeUpdate) ISING_SP_I(kModeUpdate);
  else if (mode == kModeRelaxed) ISING_SP_I(kModeRelaxed);
  else if (mode == kModeEnergy) ISING_SP_I(kModeEnergy);
  else ISING_SP_V(kModeCoupling, true);
#undef ISING_SP_I
#undef ISING_SP_V
#undef ISING_SP_ARGS
#undef ISING_SP
  ISING_CUDA(ctx, cudaGetLastError());
  return ISING_OK;
}

}  // namespace ising
