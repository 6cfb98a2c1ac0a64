// K2p: the plain FP32 form of the fused domain-selection step (Sec. III-B)
// on the CUDA cores. G = J S is a tiled SIMT SGEMM (128 spins x 128 restarts
// per block, K chunks of 16 staged in shared memory, 8 x 8 outputs per
// thread); the epilogue does, per element: loss field F = cQ G + cH h - mu s,
// gradient g = cos(theta) F, Adam, projection, rounding of the new spin, and
// the energy partials of the input spins for this block's 128 rows. In the
// relaxed mode the product runs on x = sin(theta) (X), the epilogue takes the
// rounded spins from Sr, writes x_{t+1} and leaves the energies to a
// kModeEnergy pass.
#include "ds_internal.cuh"

namespace ising {
namespace {

constexpr int BM = 128, BN = 128, BK = 16;

__global__ void to_float_kernel(const void* J, int dt, int64_t count, float* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (float)load_as_double(J, dt, e);
}

template <int MODE, bool INT_E>
__global__ void __launch_bounds__(256) plain_step_kernel(
    const float* __restrict__ J, int64_t n, int64_t B, const float* __restrict__ S,
    const float* __restrict__ Sr, float* __restrict__ Xnext,
    float* __restrict__ Snext, float* __restrict__ theta, float* __restrict__ m,
    float* __restrict__ v, const float* __restrict__ hf, const int32_t* __restrict__ hint,
    StepConsts k, const float2* __restrict__ bias, const long long* __restrict__ counters,
    long long* __restrict__ qpart, long long* __restrict__ hpart, float* __restrict__ epart,
    float* __restrict__ Gout, const int* __restrict__ live32, unsigned long long* __restrict__ work) {
  constexpr bool UPDATE = MODE == kModeUpdate || MODE == kModeRelaxed;
  constexpr bool PARTIALS = MODE == kModeUpdate || MODE == kModeEnergy;
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  const int64_t ne = n0 + BN < B ? n0 + BN : B;
  if (MODE != kModeCoupling && restarts_retired(live32, n0, ne)) return;  // (uniform per block)
  if (UPDATE && work && blockIdx.x == 0 && tid == 0) atomicAdd(work, (unsigned long long)(ne - n0));
  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;

  for (int64_t k0 = 0; k0 < n; k0 += BK) {
#pragma unroll
    for (int e = 0; e < (BM * BK) / 256; ++e) {
      int idx = tid + 256 * e;
      int row = idx / BK, kk = idx % BK;
      int64_t gi = m0 + row, gk = k0 + kk;
      As[kk][row] = (gi < n && gk < n) ? J[gi * n + gk] : 0.f;
      int64_t gb = n0 + row;
      Bs[kk][row] = (gb < B && gk < n) ? S[gb * n + gk] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[8], b[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) a[r] = As[kk][tx + 16 * r];
#pragma unroll
      for (int c = 0; c < 8; ++c) b[c] = Bs[kk][ty + 16 * c];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }

  const long long t = counters[0] + 1;
  const float2 bc = bias[t];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int64_t b = n0 + ty + 16 * c;
    int qs = 0, hs = 0;
    float es = 0.f;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int64_t i = m0 + tx + 16 * r;
      if (i < n && b < B) {
        const int64_t idx = b * n + i;
        const float G = acc[r][c];
        if (MODE == kModeCoupling) {
          Gout[idx] = G;
          continue;
        }
        const float s = Sr[idx];
        const float h = hf[i];
        if (INT_E) {
          qs += (int)s * __float2int_rn(G);
          hs += (int)s * hint[i];
        } else {
          es += s * fmaf(k.cq, G, k.ch * h);
        }
        if (UPDATE) {
          const float F = fmaf(k.cq, G, fmaf(k.ch, h, -k.mu * s));
          float th = theta[idx];
          const float g = cos_proj(th) * F;
          float mm = m[idx], vv = v[idx];
          th = adam_update(k, bc.x, bc.y, g, th, mm, vv);
          theta[idx] = th;
          m[idx] = mm;
          v[idx] = vv;
          Snext[idx] = sin_nonneg(th) ? 1.f : -1.f;
          if (MODE == kModeRelaxed) Xnext[idx] = sin_proj(th);
        }
      }
    }
    // reduce over the 16 lanes (tx) that share this column
#pragma unroll
    for (int o = 8; o; o >>= 1) {
      if (INT_E) {
        qs += __shfl_xor_sync(0xffffffffu, qs, o);
        hs += __shfl_xor_sync(0xffffffffu, hs, o);
      } else {
        es += __shfl_xor_sync(0xffffffffu, es, o);
      }
    }
    if (PARTIALS && tx == 0 && b < B) {
      const int64_t o = (int64_t)blockIdx.x * B + b;
      if (INT_E) {
        qpart[o] = qs;
        hpart[o] = hs;
      } else {
        epart[o] = es;
      }
    }
  }
}

}  // namespace

int plain_setup(ising_ds* ds) {
  ising_ctx* ctx = ds->ctx;
  ds->ld = ds->n;
  ds->Bp = ds->B;
  ds->spin_kind = kSpinF32;
  ds->mtiles = ceil_div_i(ds->n, BM);
  const int64_t nn = ds->n * ds->n;
  ISING_TRY(dev_alloc(ctx, ds->Jf, nn * 4));
  int g = (int)std::min<int64_t>((nn + 255) / 256, (int64_t)ctx->sm_count * 16);
  to_float_kernel<<<g, 256, 0, ctx->stream>>>(ds->inst.J.p, ds->inst.j_dtype, nn, ds->Jf.as<float>());
  ISING_CUDA(ctx, cudaGetLastError());
  return ISING_OK;
}

int plain_step(ising_ds* ds, int mode, float* Gout) {
  ising_ctx* ctx = ds->ctx;
  const int64_t t = ds->t + 1;
  const float* S = ds->spins[t % 3].as<float>();
  float* Sn = ds->spins[(t + 1) % 3].as<float>();
  // relaxed mode: the product's operand is x_t, the rounded spins come along
  const bool rel = mode == kModeRelaxed;
  const float* X = rel ? ds->xbuf[t % 2].as<float>() : S;
  float* Xn = rel ? ds->xbuf[(t + 1) % 2].as<float>() : nullptr;
  const int ps = (int)(t % 2);
  dim3 grid(ceil_div_i(ds->n, BM), ceil_div_i(ds->B, BN));
#define ISING_PLAIN(U, I)                                                                     \
  plain_step_kernel<U, I><<<grid, 256, 0, ctx->stream>>>(                                     \
      ds->Jf.as<float>(), ds->n, ds->B, X, S, Xn, Sn, ds->theta.as<float>(), ds->m.as<float>(),\
      ds->v.as<float>(), ds->hf.as<float>(), ds->hint.as<int32_t>(), ds->k,                   \
      ds->bias.as<float2>(), ds->counters.as<long long>(), ds->qpart[ps].as<long long>(),     \
      ds->hpart[ps].as<long long>(), ds->epart[ps].as<float>(), Gout,                        \
      ds->live.p ? ds->live.as<int>() : nullptr, ds->work.as<unsigned long long>())
  if (mode == kModeUpdate) {
    if (ds->int_energy) ISING_PLAIN(kModeUpdate, true); else ISING_PLAIN(kModeUpdate, false);
  } else if (mode == kModeEnergy) {
    if (ds->int_energy) ISING_PLAIN(kModeEnergy, true); else ISING_PLAIN(kModeEnergy, false);
  } else if (rel) {
    if (ds->int_energy) ISING_PLAIN(kModeRelaxed, true); else ISING_PLAIN(kModeRelaxed, false);
  } else {
    ISING_PLAIN(kModeCoupling, true);
  }
#undef ISING_PLAIN
  ISING_CUDA(ctx, cudaGetLastError());
  return ISING_OK;
}

}  // namespace ising
