// K3: energy of rounded spin vectors, E(s) = cQ s^T J s + cH h^T s (Sec. II).
//
// One block handles 64 rows of one vector: a warp forms (J s)_i for 8 rows
// (lanes stride over the columns of a dense row or the entries of a CSR row),
// then the block adds s_i (J s)_i and h_i s_i over its rows in a fixed order.
// A second kernel adds the block partials of each vector in index order, so
// results are deterministic. Integer couplings accumulate in int64 (exact);
// other couplings in FP64.
#include "common.cuh"

namespace ising {
namespace {

constexpr int kRowsPerBlock = 64;

template <bool INT>
__global__ void __launch_bounds__(256) energy_rows(InstView in, const int8_t* __restrict__ spins,
                                                   int h_shift, int64_t nchunks,
                                                   void* __restrict__ qpart,
                                                   void* __restrict__ hpart) {
  using Acc = typename std::conditional<INT, long long, double>::type;
  const int64_t n = in.n;
  const int64_t vec = blockIdx.y;
  const int8_t* s = spins + vec * n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ Acc sq[8], sh[8];
  Acc q_acc = 0, h_acc = 0;
  for (int r = 0; r < kRowsPerBlock / 8; ++r) {
    int64_t i = (int64_t)blockIdx.x * kRowsPerBlock + warp * (kRowsPerBlock / 8) + r;
    if (i >= n) break;
    Acc dot = 0;
    if (in.layout == ISING_LAYOUT_DENSE) {
      const int64_t base = i * n;
      for (int64_t j = lane; j < n; j += 32) {
        if (INT) dot += (Acc)load_as_int(in.J, in.j_dtype, base + j) * s[j];
        else dot += load_as_double(in.J, in.j_dtype, base + j) * (double)s[j];
      }
    } else {
      for (int64_t k = in.rowptr[i] + lane; k < in.rowptr[i + 1]; k += 32) {
        int32_t j = in.indices[k];
        if (INT) dot += (Acc)load_as_int(in.J, in.j_dtype, k) * s[j];
        else dot += load_as_double(in.J, in.j_dtype, k) * (double)s[j];
      }
    }
    for (int o = 16; o; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    if (lane == 0) {
      q_acc += dot * (Acc)s[i];
      if (in.h) {
        if (INT) h_acc += (Acc)llrint(ldexp(load_as_double(in.h, in.h_dtype, i), h_shift)) * s[i];
        else h_acc += load_as_double(in.h, in.h_dtype, i) * (double)s[i];
      }
    }
  }
  if (lane == 0) {
    sq[warp] = q_acc;
    sh[warp] = h_acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Acc a = 0, b = 0;
    for (int w = 0; w < 8; ++w) { a += sq[w]; b += sh[w]; }
    static_cast<Acc*>(qpart)[vec * nchunks + blockIdx.x] = a;
    static_cast<Acc*>(hpart)[vec * nchunks + blockIdx.x] = b;
  }
}

template <bool INT>
__global__ void energy_finish(int64_t count, int64_t nchunks, const void* __restrict__ qpart,
                              const void* __restrict__ hpart, double cq, double ch, int h_shift,
                              double* __restrict__ E, int64_t* __restrict__ Q,
                              int64_t* __restrict__ H) {
  using Acc = typename std::conditional<INT, long long, double>::type;
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= count) return;
  Acc a = 0, b = 0;
  for (int64_t c = 0; c < nchunks; ++c) {
    a += static_cast<const Acc*>(qpart)[v * nchunks + c];
    b += static_cast<const Acc*>(hpart)[v * nchunks + c];
  }
  if (INT) {
    E[v] = cq * (double)a + ch * ldexp((double)b, -h_shift);
    if (Q) Q[v] = (int64_t)a;
    if (H) H[v] = (int64_t)b;
  } else {
    E[v] = cq * (double)a + ch * (double)b;
  }
}

}  // namespace

int energy_device(ising_ctx* ctx, const DevInstance& inst, const int8_t* spins, int64_t count,
                  double* E, int64_t* Q, int64_t* H) {
  if (count <= 0) return ISING_OK;
  const bool exact = inst.j_integer && inst.j_absmax < 2147483648.0 && inst.h_dyadic;
  const int64_t nchunks = (inst.n + kRowsPerBlock - 1) / kRowsPerBlock;
  if (count > 65535) return fail(ctx, ISING_EINVAL, "energy: count > 65535 per call");
  DevMem qp, hp;
  ISING_TRY(dev_alloc(ctx, qp, (size_t)(count * nchunks) * 8));
  ISING_TRY(dev_alloc(ctx, hp, (size_t)(count * nchunks) * 8));
  dim3 grid((unsigned)nchunks, (unsigned)count);
  InstView v = view(inst);
  if (exact) {
    energy_rows<true><<<grid, 256, 0, ctx->stream>>>(v, spins, inst.h_shift, nchunks, qp.p, hp.p);
    energy_finish<true><<<ceil_div_i(count, 128), 128, 0, ctx->stream>>>(
        count, nchunks, qp.p, hp.p, inst.cq, inst.ch, inst.h_shift, E, Q, H);
  } else {
    energy_rows<false><<<grid, 256, 0, ctx->stream>>>(v, spins, 0, nchunks, qp.p, hp.p);
    energy_finish<false><<<ceil_div_i(count, 128), 128, 0, ctx->stream>>>(
        count, nchunks, qp.p, hp.p, inst.cq, inst.ch, 0, E, nullptr, nullptr);
  }
  ISING_CUDA(ctx, cudaGetLastError());
  // the scratch buffers are freed when this function returns: wait for the kernels
  ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ISING_OK;
}

}  // namespace ising
