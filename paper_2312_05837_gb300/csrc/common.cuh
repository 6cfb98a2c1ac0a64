// Internal definitions shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ising_ds.h"

struct ising_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  size_t smem_optin = 0;
  std::string err;
};

#include <nvtx3/nvToolsExt.h>

namespace ising {

// NVTX range for the duration of a scope (shows the stages of a call on a
// profiler's timeline; costs nothing without a profiler attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Records a formatted error on the context and returns `code`.
inline int fail(ising_ctx* ctx, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  return code;
}

#define ISING_CUDA(ctx, expr)                                                   \
  do {                                                                          \
    cudaError_t e_ = (expr);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      return ::ising::fail((ctx), e_ == cudaErrorMemoryAllocation ? ISING_ENOMEM \
                                                                  : ISING_ECUDA, \
                           "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                           __FILE__, __LINE__);                                 \
    }                                                                           \
  } while (0)

#define ISING_TRY(expr)        \
  do {                         \
    int r_ = (expr);           \
    if (r_ != ISING_OK) return r_; \
  } while (0)

// Owning device allocation from the stream-ordered pool: allocated and freed
// on the stream the work using it is issued on, so releasing a buffer never
// synchronises the device and repeated solves reuse pooled memory.
struct DevMem {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  DevMem() = default;
  DevMem(const DevMem&) = delete;
  DevMem& operator=(const DevMem&) = delete;
  DevMem(DevMem&& o) noexcept : p(o.p), bytes(o.bytes), stream(o.stream) { o.p = nullptr; o.bytes = 0; }
  DevMem& operator=(DevMem&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      bytes = o.bytes;
      stream = o.stream;
      o.p = nullptr;
      o.bytes = 0;
    }
    return *this;
  }
  ~DevMem() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, stream);
    p = nullptr;
    bytes = 0;
  }
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// Copies `bytes` of host memory to device memory `dst` in the order of the
// context's stream; the host buffer may go away on return. Up to 480 KB the
// bytes travel as kernel parameters (copied when each launch is queued), so
// nothing waits for the stream's earlier work (a copy from pageable memory
// first waits for the stream); larger tables are copied and waited for.
int upload_async(ising_ctx* ctx, void* dst, const void* src, size_t bytes);

inline int dev_alloc(ising_ctx* ctx, DevMem& m, size_t bytes) {
  m.release();
  if (bytes == 0) bytes = 16;
  m.stream = ctx->stream;
  cudaError_t e = cudaMallocAsync(&m.p, bytes, m.stream);
  if (e != cudaSuccess) {
    m.p = nullptr;
    cudaGetLastError();
    return fail(ctx, ISING_ENOMEM, "cudaMallocAsync(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  m.bytes = bytes;
  return ISING_OK;
}

inline int ceil_div_i(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

inline double bits_to_double(unsigned long long b) {
  double d;
  memcpy(&d, &b, sizeof d);
  return d;
}

// Energy coefficients: E(s) = cQ s^T J s + cH h^T s.
inline void coefficients(const ising_instance* in, double* cq, double* ch) {
  if (in->convention == ISING_CONV_PAPER) {
    *cq = in->j_scale;
    *ch = 1.0;
  } else {
    *cq = -0.5 * in->j_scale;
    *ch = -1.0;
  }
}

inline size_t dtype_size(int dt) {
  switch (dt) {
    case ISING_F64: return 8;
    case ISING_F32: return 4;
    case ISING_I8: return 1;
    case ISING_I32: return 4;
  }
  return 0;
}

// A validated instance copied to the device in its stored dtype, with the
// facts the solver paths need.
struct DevInstance {
  int64_t n = 0;
  int layout = ISING_LAYOUT_DENSE;
  int j_dtype = ISING_F32;
  int h_dtype = ISING_F64;
  bool has_h = false;
  int64_t nnz = 0;
  double j_scale = 1.0;
  int convention = ISING_CONV_PHYSICS;
  double cq = 0.0, ch = 0.0;
  DevMem J;       // dense n*n or nnz values, stored dtype
  DevMem indptr;  // int64 n+1
  DevMem rowptr;  // int32 n+1 (CSR)
  DevMem indices; // int32 nnz
  DevMem h;       // n, h_dtype
  // Integer facts (computed on the device at upload):
  bool j_integer = false;   // every J value is an integer
  double j_absmax = 0.0;    // max |J|
  bool h_dyadic = true;     // every h * 2^h_shift is an integer of |.| < 2^30
  int h_shift = 0;
  double h_absmax = 0.0;
};

// Uploads / copies `in` to the device and validates it (symmetry, zero
// diagonal, CSR structure; skipped when `validate` is false, for instances the
// library derived itself). Value facts are always gathered. Defined in
// instance.cu.
int upload_instance(ising_ctx* ctx, const ising_instance* in, DevInstance* out,
                    bool validate = true);

// Device view of an instance for kernels.
struct InstView {
  int64_t n;
  int layout;
  int j_dtype;
  int h_dtype;
  const void* J;
  const int32_t* rowptr;
  const int32_t* indices;
  const void* h;  // nullable
};

inline InstView view(const DevInstance& d) {
  InstView v;
  v.n = d.n;
  v.layout = d.layout;
  v.j_dtype = d.j_dtype;
  v.h_dtype = d.h_dtype;
  v.J = d.J.p;
  v.rowptr = d.rowptr.as<int32_t>();
  v.indices = d.indices.as<int32_t>();
  v.h = d.has_h ? d.h.p : nullptr;
  return v;
}

__device__ __forceinline__ double load_as_double(const void* p, int dt, int64_t i) {
  switch (dt) {
    case ISING_F64: return static_cast<const double*>(p)[i];
    case ISING_F32: return (double)static_cast<const float*>(p)[i];
    case ISING_I8: return (double)static_cast<const int8_t*>(p)[i];
    default: return (double)static_cast<const int32_t*>(p)[i];
  }
}

__device__ __forceinline__ int32_t load_as_int(const void* p, int dt, int64_t i) {
  switch (dt) {
    case ISING_I8: return (int32_t) static_cast<const int8_t*>(p)[i];
    case ISING_I32: return static_cast<const int32_t*>(p)[i];
    case ISING_F32: return (int32_t) static_cast<const float*>(p)[i];
    default: return (int32_t) static_cast<const double*>(p)[i];
  }
}

// Energy of all `count` spin vectors (K3); defined in energy.cu. spins and
// outputs are device pointers. E = cQ Q + cH H.
int energy_device(ising_ctx* ctx, const DevInstance& inst, const int8_t* spins,
                  int64_t count, double* E, int64_t* Q, int64_t* H);

// SplitMix64 output number `counter` from `seed` (Steele, Lea, Flood 2014).
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace ising
