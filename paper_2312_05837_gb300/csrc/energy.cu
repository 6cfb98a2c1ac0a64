// K3: energy of rounded spin vectors, E(s) = cQ s^T J s + cH h^T s (Sec. II).
//
// One block handles 64 rows of one vector: a warp forms (J s)_i for 8 rows
// (lanes stride over the columns of a dense row or the entries of a CSR row),
// then the block adds s_i (J s)_i and h_i s_i over its rows in a fixed order.
// A second kernel adds the block partials of each vector in index order, so
// results are deterministic. Integer couplings accumulate in int64 (exact);
// other couplings in FP64.
#include "common.cuh"

#include <atomic>

namespace ising {
namespace {

constexpr int kRowsPerBlock = 64;

// The instance as the rows kernel reads it: dense or CSR J with row offsets
// of type Off (the library's own int32 copy, or a caller's int64 offsets),
// and h scaled by 2^h_shift to integers in the exact mode.
template <typename Off>
struct RowsView {
  int64_t n;
  int layout, j_dtype, h_dtype, h_shift;
  const void* J;
  const Off* rowptr;
  const int32_t* indices;
  const void* h;  // nullable
};

template <bool INT, typename Off>
__global__ void __launch_bounds__(256) energy_rows(RowsView<Off> in, const int8_t* __restrict__ spins,
                                                   int64_t nchunks, void* __restrict__ qpart,
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
      for (int64_t k = (int64_t)in.rowptr[i] + lane; k < (int64_t)in.rowptr[i + 1]; k += 32) {
        int32_t j = in.indices[k];
        if (INT) dot += (Acc)load_as_int(in.J, in.j_dtype, k) * s[j];
        else dot += load_as_double(in.J, in.j_dtype, k) * (double)s[j];
      }
    }
    for (int o = 16; o; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    if (lane == 0) {
      q_acc += dot * (Acc)s[i];
      if (in.h) {
        if (INT) h_acc += (Acc)llrint(ldexp(load_as_double(in.h, in.h_dtype, i), in.h_shift)) * s[i];
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
  const InstView iv = view(inst);
  RowsView<int32_t> v{iv.n, iv.layout, iv.j_dtype, iv.h_dtype, exact ? inst.h_shift : 0,
                      iv.J, iv.rowptr, iv.indices, iv.h};
  if (exact) {
    energy_rows<true><<<grid, 256, 0, ctx->stream>>>(v, spins, nchunks, qp.p, hp.p);
    energy_finish<true><<<ceil_div_i(count, 128), 128, 0, ctx->stream>>>(
        count, nchunks, qp.p, hp.p, inst.cq, inst.ch, inst.h_shift, E, Q, H);
  } else {
    energy_rows<false><<<grid, 256, 0, ctx->stream>>>(v, spins, nchunks, qp.p, hp.p);
    energy_finish<false><<<ceil_div_i(count, 128), 128, 0, ctx->stream>>>(
        count, nchunks, qp.p, hp.p, inst.cq, inst.ch, 0, E, nullptr, nullptr);
  }
  ISING_CUDA(ctx, cudaGetLastError());
  // the scratch buffers are freed when this function returns: wait for the kernels
  ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ISING_OK;
}

}  // namespace ising

// ---------------------------------------------------------------------------
// Energy with no allocation at all, for callers that cannot allocate device
// memory (a host that hands the library fixed buffers, or code running where
// cudaMalloc is not allowed, such as inside a stream being captured into a
// CUDA graph by someone else). The per-block partial sums live in one
// file-scope device array instead of a cudaMalloc'd buffer.

namespace ising {
namespace {

// Scratch for the no-allocation energy: 2 MiB per device, held by every GPU
// that loads this library until the process exits. One call needs
// count * ceil(n / 64) * 16 bytes of it.
constexpr size_t kNoAllocScratchBytes = size_t(2) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device, looked up by the first call
// made with that device current (the array's host-side name is not a device
// address). Threads racing on a first call store the same address; the slots
// are atomic so that the race is well defined. A device reset invalidates
// the cached address (the library does not reset devices).
constexpr int kMaxDevices = 64;
std::atomic<void*> g_noalloc_ptr[kMaxDevices];
thread_local char g_noalloc_err[256] = "";

int noalloc_fail(int code, const char* msg) {
  snprintf(g_noalloc_err, sizeof g_noalloc_err, "%s", msg);
  return code;
}

}  // namespace
}  // namespace ising

extern "C" const char* ising_energy_noalloc_error(void) { return ising::g_noalloc_err; }

extern "C" int ising_energy_noalloc(const ising_instance* inst, const int8_t* spins,
                                    int64_t count, double* E_out, void* stream) {
  using namespace ising;
  if (!inst || !spins || !E_out) return noalloc_fail(ISING_EINVAL, "inst, spins and E_out are required");
  if (inst->mem != ISING_MEM_DEVICE)
    return noalloc_fail(ISING_EINVAL, "the instance must be in device memory");
  if (inst->n < 1) return noalloc_fail(ISING_EINVAL, "n must be >= 1");
  if (inst->layout != ISING_LAYOUT_DENSE && inst->layout != ISING_LAYOUT_CSR)
    return noalloc_fail(ISING_EINVAL, "unknown layout");
  if (dtype_size(inst->j_dtype) == 0 || !inst->J) return noalloc_fail(ISING_EINVAL, "bad J");
  if (inst->layout == ISING_LAYOUT_CSR && (!inst->indptr || (!inst->indices && inst->nnz > 0)))
    return noalloc_fail(ISING_EINVAL, "CSR needs indptr and indices");
  if (inst->h && (dtype_size(inst->h_dtype) == 0 || inst->h_dtype == ISING_I8))
    return noalloc_fail(ISING_EINVAL, "h_dtype must be F64, F32 or I32");
  if (count < 0 || count > 65535) return noalloc_fail(ISING_EINVAL, "count must lie in [0, 65535]");
  if (count == 0) return ISING_OK;
  const int64_t nchunks = (inst->n + kRowsPerBlock - 1) / kRowsPerBlock;
  const size_t need = (size_t)count * (size_t)nchunks * 16;
  if (need > kNoAllocScratchBytes)
    return noalloc_fail(ISING_EINVAL,
                        "count * ceil(n / 64) * 16 bytes exceeds the 2 MiB no-allocation scratch");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return noalloc_fail(ISING_ECUDA, "no current CUDA device");
  }
  void* sp = g_noalloc_ptr[dev].load(std::memory_order_acquire);
  if (!sp) {
    cudaError_t e = cudaGetSymbolAddress(&sp, g_noalloc_scratch);
    if (e != cudaSuccess || !sp) {
      cudaGetLastError();
      return noalloc_fail(ISING_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
    }
    g_noalloc_ptr[dev].store(sp, std::memory_order_release);
  }
  unsigned char* scratch = static_cast<unsigned char*>(sp);
  void* qp = scratch;
  void* hp = scratch + (size_t)count * nchunks * 8;
  const bool exact = (inst->j_dtype == ISING_I8 || inst->j_dtype == ISING_I32) &&
                     (!inst->h || inst->h_dtype == ISING_I32);
  double cq, ch;
  coefficients(inst, &cq, &ch);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  dim3 grid((unsigned)nchunks, (unsigned)count);
  // integer h (I32) enters the exact sums unscaled
  const RowsView<int64_t> v{inst->n, inst->layout, inst->j_dtype, inst->h_dtype, 0, inst->J,
                            inst->indptr, inst->indices, inst->h};
  if (exact) {
    energy_rows<true><<<grid, 256, 0, st>>>(v, spins, nchunks, qp, hp);
    energy_finish<true><<<(unsigned)((count + 127) / 128), 128, 0, st>>>(
        count, nchunks, qp, hp, cq, ch, 0, E_out, nullptr, nullptr);
  } else {
    energy_rows<false><<<grid, 256, 0, st>>>(v, spins, nchunks, qp, hp);
    energy_finish<false><<<(unsigned)((count + 127) / 128), 128, 0, st>>>(
        count, nchunks, qp, hp, cq, ch, 0, E_out, nullptr, nullptr);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(ISING_ECUDA, cudaGetErrorString(e));
  return ISING_OK;
}
