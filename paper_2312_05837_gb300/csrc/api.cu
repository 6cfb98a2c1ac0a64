// Context management, the energy call (K3) and the full solve
// (pruning -> domain selection -> reconstruction -> energy).
#include "common.cuh"
#include "tcgen05.cuh"

#include <algorithm>
#include <cstring>

using namespace ising;

extern "C" int ising_version(void) { return 10000; }

namespace ising {

// One launch carries up to kUploadBytes (kernel parameters may take up to
// 32764 bytes in all).
constexpr int kUploadBytes = 30720;
struct UploadChunk {
  unsigned char* dst;
  int len;
  unsigned char bytes[kUploadBytes];
};

__global__ void upload_kernel(const UploadChunk c) {
  for (int i = threadIdx.x; i < c.len; i += blockDim.x) c.dst[i] = c.bytes[i];
}

int upload_async(ising_ctx* ctx, void* dst, const void* src, size_t bytes) {
  static_assert(sizeof(UploadChunk) <= 32764, "kernel parameter limit");
  if (bytes > 16 * (size_t)kUploadBytes) {
    // large: one copy, then a wait for it (the host buffer goes away on return)
    ISING_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return ISING_OK;
  }
  const unsigned char* s = static_cast<const unsigned char*>(src);
  unsigned char* d = static_cast<unsigned char*>(dst);
  UploadChunk* c = new UploadChunk;
  for (size_t off = 0; off < bytes; off += kUploadBytes) {
    const int len = (int)std::min<size_t>(kUploadBytes, bytes - off);
    c->dst = d + off;
    c->len = len;
    memcpy(c->bytes, s + off, len);
    upload_kernel<<<1, 256, 0, ctx->stream>>>(*c);
  }
  delete c;
  ISING_CUDA(ctx, cudaGetLastError());
  return ISING_OK;
}

}  // namespace ising

extern "C" int ising_create(ising_ctx** out, int device, void* stream) {
  if (!out) return ISING_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return ISING_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return ISING_ECUDA;
  auto ctx = new ising_ctx();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(stream);
  int sms = 0, optin = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  ctx->sm_count = std::max(sms, 1);
  ctx->smem_optin = (size_t)optin;
  // keep freed pool memory cached for the next solve instead of returning it
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  *out = ctx;
  return ISING_OK;
}

extern "C" int ising_destroy(ising_ctx* ctx) {
  if (!ctx) return ISING_OK;
  cudaStreamSynchronize(ctx->stream);
  delete ctx;
  return ISING_OK;
}

extern "C" const char* ising_last_error(const ising_ctx* ctx) {
  return ctx ? ctx->err.c_str() : "null context";
}

extern "C" int ising_set_stream(ising_ctx* ctx, void* stream) {
  if (!ctx) return ISING_EINVAL;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return ISING_OK;
}

extern "C" int ising_synchronize(ising_ctx* ctx) {
  if (!ctx) return ISING_EINVAL;
  ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ISING_OK;
}

extern "C" int ising_energy(ising_ctx* ctx, const ising_instance* inst, const int8_t* spins,
                            int64_t count, double* E_out, int64_t* Q_out, int64_t* H_out,
                            int mem) {
  if (!ctx) return ISING_EINVAL;
  if (count < 0) return fail(ctx, ISING_EINVAL, "count must be >= 0");
  if (count > 0 && (!spins || !E_out)) return fail(ctx, ISING_EINVAL, "spins and E_out are required");
  if (mem != ISING_MEM_HOST && mem != ISING_MEM_DEVICE) return fail(ctx, ISING_EINVAL, "bad mem");
  ISING_CUDA(ctx, cudaSetDevice(ctx->device));
  DevInstance I;
  ISING_TRY(upload_instance(ctx, inst, &I));
  const bool exact = I.j_integer && I.j_absmax < 2147483648.0 && I.h_dyadic;
  if ((Q_out || H_out) && !exact)
    return fail(ctx, ISING_EINVAL, "Q/H outputs need an integer instance");
  if (H_out && I.h_shift != 0) return fail(ctx, ISING_EINVAL, "H output needs an integer h");
  if (count == 0) return ISING_OK;
  cudaStream_t st = ctx->stream;
  const int64_t n = I.n;
  DevMem s, E, Q, H;
  const int8_t* sp = spins;
  if (mem == ISING_MEM_HOST) {
    ISING_TRY(dev_alloc(ctx, s, (size_t)count * n));
    ISING_CUDA(ctx, cudaMemcpyAsync(s.p, spins, (size_t)count * n, cudaMemcpyHostToDevice, st));
    sp = s.as<int8_t>();
  }
  ISING_TRY(dev_alloc(ctx, E, count * 8));
  ISING_TRY(dev_alloc(ctx, Q, count * 8));
  ISING_TRY(dev_alloc(ctx, H, count * 8));
  for (int64_t c0 = 0; c0 < count; c0 += 65535) {
    int64_t c = std::min<int64_t>(65535, count - c0);
    ISING_TRY(energy_device(ctx, I, sp + c0 * n, c, E.as<double>() + c0,
                            exact ? Q.as<int64_t>() + c0 : nullptr,
                            exact ? H.as<int64_t>() + c0 : nullptr));
  }
  cudaMemcpyKind k = mem == ISING_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  ISING_CUDA(ctx, cudaMemcpyAsync(E_out, E.p, count * 8, k, st));
  if (Q_out) ISING_CUDA(ctx, cudaMemcpyAsync(Q_out, Q.p, count * 8, k, st));
  if (H_out) ISING_CUDA(ctx, cudaMemcpyAsync(H_out, H.p, count * 8, k, st));
  ISING_CUDA(ctx, cudaStreamSynchronize(st));
  return ISING_OK;
}

namespace {

// Two bounded waits that nothing completes (see ising_selftest_waits).
__global__ void selftest_wait_kernel(const unsigned int* flag, long long limit, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    ising::tc::mbar_init(&bar, 1);
    ising::tc::fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  int gave_up = 0;
  if (!ising::tc::mbar_wait(&bar, 0, nullptr, limit)) gave_up |= 1;
  const long long c0 = clock64();
  while (ising::tc::ld_acquire_gpu(flag) == 0u) {
    if (clock64() - c0 > limit) {
      gave_up |= 2;
      break;
    }
  }
  *status = gave_up;
}

}  // namespace

extern "C" int ising_selftest_waits(ising_ctx* ctx, int64_t limit_cycles, int32_t* gave_up) {
  if (!ctx) return ISING_EINVAL;
  if (limit_cycles < 1 || limit_cycles > (int64_t(1) << 34))
    return fail(ctx, ISING_EINVAL, "limit_cycles must lie in [1, 2^34]");
  ISING_CUDA(ctx, cudaSetDevice(ctx->device));
  DevMem buf;
  ISING_TRY(dev_alloc(ctx, buf, 16));
  ISING_CUDA(ctx, cudaMemsetAsync(buf.p, 0, 16, ctx->stream));
  selftest_wait_kernel<<<1, 32, 0, ctx->stream>>>(buf.as<unsigned int>(), (long long)limit_cycles,
                                                  buf.as<int>() + 1);
  ISING_CUDA(ctx, cudaGetLastError());
  int st = 0;
  ISING_CUDA(ctx, cudaMemcpyAsync(&st, buf.as<int>() + 1, 4, cudaMemcpyDeviceToHost, ctx->stream));
  ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (gave_up) *gave_up = st;
  if (st) return fail(ctx, ISING_ETIMEOUT, "bounded waits gave up (mask %d)", st);
  return ISING_OK;
}

namespace ising {
int prune_device(ising_ctx* ctx, const DevInstance& I, int flags, ising_prune_result** out);
int ds_create_impl(ising_ctx* ctx, const ising_instance* inst, const ising_ds_params* p,
                   ising_ds** out, bool validate);
}

// The instance is uploaded and validated once; domain selection runs on the
// reduced instance the library derived from it, and the final energy is taken
// on the uploaded copy.
extern "C" int ising_solve(ising_ctx* ctx, const ising_instance* inst, const ising_ds_params* p,
                           int prune_flags, int8_t* best_spins, double* best_energy,
                           ising_ds_stats* stats, int mem) {
  if (!ctx) return ISING_EINVAL;
  if (!inst) return fail(ctx, ISING_EINVAL, "instance is NULL");
  if (mem != ISING_MEM_HOST && mem != ISING_MEM_DEVICE) return fail(ctx, ISING_EINVAL, "bad mem");
  if (prune_flags & ~ISING_PRUNE_ZERO_RULE) return fail(ctx, ISING_EINVAL, "unknown prune flags");
  if (!p) return fail(ctx, ISING_EINVAL, "params is NULL");
  ISING_CUDA(ctx, cudaSetDevice(ctx->device));
  NvtxRange range("ising_solve");
  cudaStream_t st = ctx->stream;
  DevInstance I;
  {
    NvtxRange r("upload+validate");
    ISING_TRY(upload_instance(ctx, inst, &I));
  }
  ising_prune_result* pr = nullptr;
  {
    NvtxRange r("prune");
    ISING_TRY(prune_device(ctx, I, prune_flags, &pr));
  }
  int64_t nG = 0;
  ising_prune_info(pr, &nG, nullptr, nullptr, nullptr, nullptr);
  const int64_t n = inst->n;
  int rc = ISING_OK;
  DevMem sG, full, E;
  ising_ds_stats ds_stats{};
  do {
    if ((rc = dev_alloc(ctx, sG, std::max<int64_t>(nG, 1))) != ISING_OK) break;
    if ((rc = dev_alloc(ctx, full, n)) != ISING_OK) break;
    if ((rc = dev_alloc(ctx, E, 8)) != ISING_OK) break;
    if (nG > 0) {
      NvtxRange r("select_domain");
      ising_instance red;
      ising_prune_reduced(pr, &red);
      double eg = 0.0;
      ising_ds* ds = nullptr;
      rc = ds_create_impl(ctx, &red, p, &ds, false);
      if (rc == ISING_OK) rc = ising_ds_finish(ds);
      if (rc == ISING_OK) rc = ising_ds_result(ds, sG.as<int8_t>(), &eg, &ds_stats, ISING_MEM_DEVICE);
      ising_ds_destroy(ds);
      if (rc != ISING_OK) break;
    }
    NvtxRange rr("reconstruct+energy");
    rc = ising_reconstruct(ctx, pr, sG.as<int8_t>(), full.as<int8_t>(), ISING_MEM_DEVICE);
    if (rc != ISING_OK) break;
    // the energy of the reconstructed spins on the full instance
    rc = energy_device(ctx, I, full.as<int8_t>(), 1, E.as<double>(), nullptr, nullptr);
    if (rc != ISING_OK) break;
    cudaMemcpyKind k = mem == ISING_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (best_spins) {
      cudaError_t e = cudaMemcpyAsync(best_spins, full.p, n, k, st);
      if (e != cudaSuccess) { rc = fail(ctx, ISING_ECUDA, "copy of spins failed"); break; }
    }
    if (best_energy) {
      cudaError_t e = cudaMemcpyAsync(best_energy, E.p, 8, k, st);
      if (e != cudaSuccess) { rc = fail(ctx, ISING_ECUDA, "copy of energy failed"); break; }
    }
    cudaStreamSynchronize(st);
    if (stats) *stats = ds_stats;
  } while (0);
  ising_prune_free(pr);
  return rc;
}
