// Upload and validation of an Ising instance (Sec. II: J real symmetric with
// zero diagonal, h real). Integer facts about J and h are gathered here so
// that the solver paths can choose exact integer energy accumulation.
#include "common.cuh"

#include <cmath>

namespace ising {
namespace {

struct ValFlags {
  unsigned int bad;             // bit 0 asymmetric, 1 diagonal, 2 CSR order/range, 3 indptr, 4 non-finite
  unsigned int j_nonint;        // some J value is not an integer
  unsigned long long j_absmax;  // bit pattern of max |J| (non-negative double)
  unsigned int h_mask;          // bit k: every h * 2^k is an integer below 2^30
  unsigned long long h_absmax;
};

// Facts gathered per thread and merged once per warp (a same-address atomic
// per element would serialise millions of updates).
struct LocalFacts {
  unsigned int bad = 0, nonint = 0;
  double absmax = 0.0;
  __device__ void note(double x) {
    if (!isfinite(x)) bad |= 16u;
    if (x != rint(x)) nonint = 1u;
    absmax = fmax(absmax, fabs(x));
  }
  __device__ void flush(ValFlags* f) {
    for (int o = 16; o; o >>= 1) {
      bad |= __shfl_xor_sync(0xffffffffu, bad, o);
      nonint |= __shfl_xor_sync(0xffffffffu, nonint, o);
      absmax = fmax(absmax, __shfl_xor_sync(0xffffffffu, absmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
      if (bad) atomicOr(&f->bad, bad);
      if (nonint) atomicOr(&f->j_nonint, nonint);
      atomicMax(&f->j_absmax, (unsigned long long)__double_as_longlong(absmax));
    }
  }
};

// Dense: J[i][j] == J[j][i] exactly, J[i][i] == 0, plus value facts. Every
// thread runs the same number of loop trips so the warp-level merge at the
// end sees all 32 lanes.
__global__ void check_dense(const void* J, int dt, int64_t n, ValFlags* f, bool structure) {
  const int64_t total = n * n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  LocalFacts lf;
  const int64_t e0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t trips = (total + stride - 1) / stride;
  for (int64_t k = 0; k < trips; ++k) {
    const int64_t e = e0 + k * stride;
    if (e >= total) continue;
    const int64_t i = e / n, j = e - i * n;
    const double x = load_as_double(J, dt, e);
    lf.note(x);
    if (!structure) continue;
    if (i == j) {
      if (x != 0.0) lf.bad |= 2u;
    } else if (j > i) {
      const double y = load_as_double(J, dt, j * n + i);
      if (!(x == y)) lf.bad |= 1u;
    }
  }
  lf.flush(f);
}

__global__ void check_indptr(const int64_t* indptr, int64_t n, int64_t nnz, int32_t* rowptr,
                             ValFlags* f) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t a = indptr[i];
    if (i == 0 && a != 0) atomicOr(&f->bad, 8u);
    if (i == n && a != nnz) atomicOr(&f->bad, 8u);
    if (i < n && indptr[i + 1] < a) atomicOr(&f->bad, 8u);
    rowptr[i] = (int32_t)a;
  }
}

// CSR rows: columns in range, strictly increasing, no diagonal; each (i,j,v)
// has a partner (j,i,v) found by binary search in row j.
__global__ void check_csr(const int64_t* indptr, const int32_t* idx, const void* vals, int dt,
                          int64_t n, ValFlags* f, bool structure) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t trips = (n + stride - 1) / stride;
  LocalFacts lf;
  for (int64_t tr = 0; tr < trips; ++tr) {
    const int64_t i = i0 + tr * stride;
    if (i >= n) continue;
    int64_t a = indptr[i], b = indptr[i + 1];
    int32_t prev = -1;
    for (int64_t k = a; k < b; ++k) {
      int32_t j = idx[k];
      double x = load_as_double(vals, dt, k);
      lf.note(x);
      if (!structure) continue;
      if (j < 0 || j >= n || j <= prev) {
        lf.bad |= 4u;
        break;
      }
      prev = j;
      if (j == i) {
        lf.bad |= 2u;
        continue;
      }
      int64_t lo = indptr[j], hi = indptr[j + 1] - 1;
      bool found = false;
      while (lo <= hi) {
        int64_t mid = (lo + hi) >> 1;
        int32_t c = idx[mid];
        if (c == (int32_t)i) {
          found = (load_as_double(vals, dt, mid) == x);
          break;
        }
        if (c < (int32_t)i) lo = mid + 1; else hi = mid - 1;
      }
      if (!found) lf.bad |= 1u;
    }
  }
  lf.flush(f);
}

__global__ void check_h(const void* h, int dt, int64_t n, ValFlags* f) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t trips = (n + stride - 1) / stride;
  unsigned int bad = 0, mask_all = 0x1FFu;
  double amax = 0.0;
  for (int64_t tr = 0; tr < trips; ++tr) {
    const int64_t i = i0 + tr * stride;
    if (i >= n) continue;
    double x = load_as_double(h, dt, i);
    if (!isfinite(x)) bad |= 16u;
    amax = fmax(amax, fabs(x));
    unsigned int mask = 0;
    for (int k = 0; k <= 8; ++k) {
      double y = ldexp(x, k);
      if (y == rint(y) && fabs(y) < 1073741824.0) mask |= 1u << k;
    }
    mask_all &= mask;
  }
  for (int o = 16; o; o >>= 1) {
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    mask_all &= __shfl_xor_sync(0xffffffffu, mask_all, o);
    amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(&f->bad, bad);
    atomicAnd(&f->h_mask, mask_all);
    atomicMax(&f->h_absmax, (unsigned long long)__double_as_longlong(amax));
  }
}

int grid_for(ising_ctx* ctx, int64_t work) {
  int64_t g = (work + 255) / 256;
  int64_t cap = (int64_t)ctx->sm_count * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

int upload_instance(ising_ctx* ctx, const ising_instance* in, DevInstance* out, bool validate) {
  if (!in) return fail(ctx, ISING_EINVAL, "instance is NULL");
  if (in->n < 1) return fail(ctx, ISING_EINVAL, "n must be >= 1 (got %lld)", (long long)in->n);
  if (in->n > (int64_t)INT32_MAX - 1) return fail(ctx, ISING_EINVAL, "n too large");
  if (in->layout != ISING_LAYOUT_DENSE && in->layout != ISING_LAYOUT_CSR)
    return fail(ctx, ISING_EINVAL, "unknown layout %d", in->layout);
  if (dtype_size(in->j_dtype) == 0) return fail(ctx, ISING_EINVAL, "unknown j_dtype %d", in->j_dtype);
  if (in->h && (dtype_size(in->h_dtype) == 0 || in->h_dtype == ISING_I8))
    return fail(ctx, ISING_EINVAL, "h_dtype must be F64, F32 or I32");
  if (in->convention != ISING_CONV_PHYSICS && in->convention != ISING_CONV_PAPER)
    return fail(ctx, ISING_EINVAL, "unknown convention %d", in->convention);
  if (in->mem != ISING_MEM_HOST && in->mem != ISING_MEM_DEVICE)
    return fail(ctx, ISING_EINVAL, "unknown mem %d", in->mem);
  if (!std::isfinite(in->j_scale)) return fail(ctx, ISING_EINVAL, "j_scale must be finite");
  if (!in->J) return fail(ctx, ISING_EINVAL, "J is NULL");
  const int64_t n = in->n;
  cudaMemcpyKind kind = in->mem == ISING_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaStream_t st = ctx->stream;
  out->n = n;
  out->layout = in->layout;
  out->j_dtype = in->j_dtype;
  out->j_scale = in->j_scale;
  out->convention = in->convention;
  coefficients(in, &out->cq, &out->ch);
  const size_t jsz = dtype_size(in->j_dtype);

  DevMem flags;
  ISING_TRY(dev_alloc(ctx, flags, sizeof(ValFlags)));
  ValFlags f0{};
  f0.h_mask = 0x1FFu;
  ISING_CUDA(ctx, cudaMemcpyAsync(flags.p, &f0, sizeof f0, cudaMemcpyHostToDevice, st));
  ValFlags* fd = flags.as<ValFlags>();

  if (in->layout == ISING_LAYOUT_DENSE) {
    if ((uint64_t)n > 46340ull) return fail(ctx, ISING_EINVAL, "dense n too large");
    size_t bytes = (size_t)n * (size_t)n * jsz;
    ISING_TRY(dev_alloc(ctx, out->J, bytes));
    ISING_CUDA(ctx, cudaMemcpyAsync(out->J.p, in->J, bytes, kind, st));
    out->nnz = n * n;
    check_dense<<<grid_for(ctx, n * n), 256, 0, st>>>(out->J.p, in->j_dtype, n, fd, validate);
    ISING_CUDA(ctx, cudaGetLastError());
  } else {
    if (!in->indptr || (!in->indices && in->nnz > 0))
      return fail(ctx, ISING_EINVAL, "CSR instance needs indptr and indices");
    if (in->nnz < 0 || in->nnz > (int64_t)INT32_MAX)
      return fail(ctx, ISING_EINVAL, "nnz out of range (%lld)", (long long)in->nnz);
    out->nnz = in->nnz;
    ISING_TRY(dev_alloc(ctx, out->J, (size_t)in->nnz * jsz));
    ISING_TRY(dev_alloc(ctx, out->indptr, (size_t)(n + 1) * 8));
    ISING_TRY(dev_alloc(ctx, out->rowptr, (size_t)(n + 1) * 4));
    ISING_TRY(dev_alloc(ctx, out->indices, (size_t)in->nnz * 4));
    if (in->nnz) {
      ISING_CUDA(ctx, cudaMemcpyAsync(out->J.p, in->J, (size_t)in->nnz * jsz, kind, st));
      ISING_CUDA(ctx, cudaMemcpyAsync(out->indices.p, in->indices, (size_t)in->nnz * 4, kind, st));
    }
    ISING_CUDA(ctx, cudaMemcpyAsync(out->indptr.p, in->indptr, (size_t)(n + 1) * 8, kind, st));
    check_indptr<<<grid_for(ctx, n + 1), 256, 0, st>>>(out->indptr.as<int64_t>(), n, in->nnz,
                                                       out->rowptr.as<int32_t>(), fd);
    ISING_CUDA(ctx, cudaGetLastError());
    ValFlags fh;
    ISING_CUDA(ctx, cudaMemcpyAsync(&fh, fd, sizeof fh, cudaMemcpyDeviceToHost, st));
    ISING_CUDA(ctx, cudaStreamSynchronize(st));
    if (fh.bad & 8u) return fail(ctx, ISING_EINVAL, "CSR indptr is not a valid offset array");
    check_csr<<<grid_for(ctx, n), 256, 0, st>>>(out->indptr.as<int64_t>(),
                                                out->indices.as<int32_t>(), out->J.p,
                                                in->j_dtype, n, fd, validate);
    ISING_CUDA(ctx, cudaGetLastError());
  }
  out->has_h = in->h != nullptr;
  out->h_dtype = in->h ? in->h_dtype : ISING_F64;
  if (in->h) {
    size_t hb = (size_t)n * dtype_size(in->h_dtype);
    ISING_TRY(dev_alloc(ctx, out->h, hb));
    ISING_CUDA(ctx, cudaMemcpyAsync(out->h.p, in->h, hb, kind, st));
    check_h<<<grid_for(ctx, n), 256, 0, st>>>(out->h.p, in->h_dtype, n, fd);
    ISING_CUDA(ctx, cudaGetLastError());
  }
  ValFlags fh;
  ISING_CUDA(ctx, cudaMemcpyAsync(&fh, fd, sizeof fh, cudaMemcpyDeviceToHost, st));
  ISING_CUDA(ctx, cudaStreamSynchronize(st));
  if (fh.bad & 16u) return fail(ctx, ISING_EINVAL, "J or h holds a non-finite value");
  if (fh.bad & 4u) return fail(ctx, ISING_EINVAL, "CSR columns out of range or not strictly increasing");
  if (fh.bad & 2u) return fail(ctx, ISING_EINVAL, "J has a non-zero diagonal");
  if (fh.bad & 1u) return fail(ctx, ISING_EINVAL, "J is not symmetric");
  out->j_integer = fh.j_nonint == 0;
  out->j_absmax = bits_to_double(fh.j_absmax);
  out->h_absmax = in->h ? bits_to_double(fh.h_absmax) : 0.0;
  out->h_dyadic = true;
  out->h_shift = 0;
  if (in->h) {
    out->h_dyadic = fh.h_mask != 0;
    for (int k = 0; k <= 8; ++k)
      if (fh.h_mask & (1u << k)) { out->h_shift = k; break; }
  }
  return ISING_OK;
}

}  // namespace ising
