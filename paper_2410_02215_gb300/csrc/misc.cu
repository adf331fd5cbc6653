// Small device kernels used by the contraction-tree executor: per-step
// max-abs normalisation with an FP64 log-scale accumulator kept on the
// device (no host round trip), and FP32 <-> FP64 casts; and the self-test of
// the kernels' bounded waits.
#include <algorithm>

#include "batch.h"
#include "ptx.cuh"

namespace ftn {

// max |x| as the ordered bits of a non-negative double (atomicMax).
template <typename T>
__global__ void maxabs_kernel(const T* __restrict__ x, int64_t n, unsigned long long* __restrict__ mx) {
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs((double)x[i]));
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(mx, (unsigned long long)__double_as_longlong(m));
}

template <typename Ti, typename To>
__global__ void cast_kernel(const Ti* __restrict__ x, To* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (To)x[i];
}

// Small tensors: one CTA finds max |x|, scales and accumulates the log; it
// also clears both max words of the large-tensor path.
template <typename T>
__device__ __forceinline__ void normalize_small_body(T* __restrict__ x, int64_t n, double* __restrict__ logacc,
                                                     unsigned long long* __restrict__ words) {
  if (threadIdx.x == 0) words[0] = words[1] = 0ull;
  __shared__ double red[32];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs((double)x[i]));
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) red[0] = m;
  }
  __syncthreads();
  m = red[0];
  if (!(m > 0.0)) return;
  const T inv = (T)(1.0 / m);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) x[i] *= inv;
  if (threadIdx.x == 0) *logacc += log(m);
}

template <typename T>
__global__ void __launch_bounds__(1024) normalize_small_kernel(T* __restrict__ x, int64_t n,
                                                                double* __restrict__ logacc,
                                                                unsigned long long* __restrict__ words) {
  normalize_small_body<T>(x, n, logacc, words);
}

// Large tensors: max |x| into word `cur` (atomicMax), then scale; the scale
// kernel clears the other word for the next step, so no separate memset.
template <typename T>
__global__ void scale2_kernel(T* __restrict__ x, int64_t n, unsigned long long* __restrict__ words, int cur,
                              double* __restrict__ logacc) {
  const double m = __longlong_as_double((long long)words[cur]);
  if (blockIdx.x == 0 && threadIdx.x == 0) words[cur ^ 1] = 0ull;
  if (!(m > 0.0)) return;
  const T inv = (T)(1.0 / m);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) *logacc += log(m);
}

static unsigned grid_for(ftn_ctx ctx, int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > (int64_t)ctx->num_sms * 8) g = (int64_t)ctx->num_sms * 8;
  return (unsigned)(g < 1 ? 1 : g);
}

// d_state layout: [0] log-scale accumulator (double), [1], [2] max words.
// `step` alternates the max word; both start zeroed.
ftn_status normalize_tensor(ftn_ctx ctx, ftn_tensor t, void* d_state, int step) {
  double* logacc = (double*)d_state;
  unsigned long long* words = (unsigned long long*)((char*)d_state + 8);
  if (t->numel == 0) return FTN_OK;
  const int cur = step & 1;
  if (t->numel <= 65536) {
    if (t->dtype == FTN_F64)
      normalize_small_kernel<double><<<1, 1024, 0, ctx->stream>>>((double*)t->data, t->numel, logacc, words);
    else
      normalize_small_kernel<float><<<1, 1024, 0, ctx->stream>>>((float*)t->data, t->numel, logacc, words);
    ctx->launches += 1;
    FTN_CUDA(cudaGetLastError());
    return FTN_OK;
  }
  const unsigned g = grid_for(ctx, t->numel);
  if (t->dtype == FTN_F64) {
    maxabs_kernel<double><<<g, 256, 0, ctx->stream>>>((const double*)t->data, t->numel, words + cur);
    scale2_kernel<double><<<g, 256, 0, ctx->stream>>>((double*)t->data, t->numel, words, cur, logacc);
  } else {
    maxabs_kernel<float><<<g, 256, 0, ctx->stream>>>((const float*)t->data, t->numel, words + cur);
    scale2_kernel<float><<<g, 256, 0, ctx->stream>>>((float*)t->data, t->numel, words, cur, logacc);
  }
  ctx->launches += 2;
  FTN_CUDA(cudaGetLastError());
  return FTN_OK;
}

ftn_status cast_tensor(ftn_ctx ctx, ftn_tensor t, ftn_dtype to, ftn_tensor* out) {
  FTN_TRY(make_tensor(ctx, t->rank, t->d0, t->d1, t->dual, t->parity, to, out));
  if (t->numel == 0) return FTN_OK;
  const unsigned g = grid_for(ctx, t->numel);
  if (t->dtype == FTN_F64 && to == FTN_F32)
    cast_kernel<double, float><<<g, 256, 0, ctx->stream>>>((const double*)t->data, (float*)(*out)->data, t->numel);
  else if (t->dtype == FTN_F32 && to == FTN_F64)
    cast_kernel<float, double><<<g, 256, 0, ctx->stream>>>((const float*)t->data, (double*)(*out)->data, t->numel);
  else
    FTN_CUDA(cudaMemcpyAsync((*out)->data, t->data, t->numel * dtype_size(to), cudaMemcpyDeviceToDevice, ctx->stream));
  ctx->launches += 1;
  FTN_CUDA(cudaGetLastError());
  return FTN_OK;
}

// ---- batched forms (many tensors per launch, the same arithmetic) ----------------

template <typename T>
__global__ void __launch_bounds__(1024) normalize_small_batch_kernel(const NormJob* __restrict__ jobs) {
  const NormJob J = jobs[blockIdx.x];
  normalize_small_body<T>(reinterpret_cast<T*>(J.x), J.n, J.logacc, J.words);
}

// job of tile t: the last job whose first tile is <= t
template <typename J>
__device__ __forceinline__ const J& find_tile_job(const J* __restrict__ jobs, int n, int64_t t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].tile_begin <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  return jobs[lo];
}

template <typename T>
__global__ void maxabs_batch_kernel(const NormJob* __restrict__ jobs, int njobs, int64_t tiles) {
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const NormJob& J = find_tile_job(jobs, njobs, t);
    const int64_t i0 = (t - J.tile_begin) * NORM_TILE;
    const int64_t i1 = i0 + NORM_TILE < J.n ? i0 + NORM_TILE : J.n;
    const T* x = reinterpret_cast<const T*>(J.x);
    double m = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) m = fmax(m, fabs((double)x[i]));
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(J.words + J.cur, (unsigned long long)__double_as_longlong(m));
  }
}

// Scales every tile by 1 / max; the job's first tile also clears the other
// max word (for the next step) and adds log(max) to the accumulator.
template <typename T>
__global__ void scale_batch_kernel(const NormJob* __restrict__ jobs, int njobs, int64_t tiles) {
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const NormJob& J = find_tile_job(jobs, njobs, t);
    const double m = __longlong_as_double((long long)J.words[J.cur]);
    const bool first = t == J.tile_begin;
    if (first && threadIdx.x == 0) J.words[J.cur ^ 1] = 0ull;
    if (!(m > 0.0)) continue;
    const int64_t i0 = (t - J.tile_begin) * NORM_TILE;
    const int64_t i1 = i0 + NORM_TILE < J.n ? i0 + NORM_TILE : J.n;
    T* x = reinterpret_cast<T*>(J.x);
    const T inv = (T)(1.0 / m);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) x[i] *= inv;
    if (first && threadIdx.x == 0) *J.logacc += log(m);
  }
}

ftn_status launch_normalize_batch(ftn_ctx ctx, ftn_dtype dt, const NormJob* d_small, int nsmall,
                                  const NormJob* d_large, int nlarge, int64_t large_tiles) {
  const bool f64 = dt == FTN_F64;
  if (nsmall > 0) {
    if (f64)
      normalize_small_batch_kernel<double><<<(unsigned)nsmall, 1024, 0, ctx->stream>>>(d_small);
    else
      normalize_small_batch_kernel<float><<<(unsigned)nsmall, 1024, 0, ctx->stream>>>(d_small);
    ctx->launches += 1;
    FTN_CUDA(cudaGetLastError());
  }
  if (nlarge > 0 && large_tiles > 0) {
    const unsigned g = (unsigned)std::min<int64_t>(large_tiles, (int64_t)ctx->num_sms * 8);
    if (f64) {
      maxabs_batch_kernel<double><<<g, 256, 0, ctx->stream>>>(d_large, nlarge, large_tiles);
      scale_batch_kernel<double><<<g, 256, 0, ctx->stream>>>(d_large, nlarge, large_tiles);
    } else {
      maxabs_batch_kernel<float><<<g, 256, 0, ctx->stream>>>(d_large, nlarge, large_tiles);
      scale_batch_kernel<float><<<g, 256, 0, ctx->stream>>>(d_large, nlarge, large_tiles);
    }
    ctx->launches += 2;
    FTN_CUDA(cudaGetLastError());
  }
  return FTN_OK;
}

template <typename Ti, typename To>
__global__ void cast_batch_kernel(const CastJob* __restrict__ jobs, int njobs, int64_t tiles) {
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const CastJob& J = find_tile_job(jobs, njobs, t);
    const int64_t i0 = (t - J.tile_begin) * CAST_TILE;
    const int64_t i1 = i0 + CAST_TILE < J.n ? i0 + CAST_TILE : J.n;
    const Ti* x = reinterpret_cast<const Ti*>(J.src);
    To* y = reinterpret_cast<To*>(J.dst);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) y[i] = (To)x[i];
  }
}

ftn_status launch_cast_batch(ftn_ctx ctx, ftn_dtype from, ftn_dtype to, const CastJob* d_jobs, int njobs,
                             int64_t tiles) {
  if (njobs == 0 || tiles == 0) return FTN_OK;
  const unsigned g = (unsigned)std::min<int64_t>(tiles, (int64_t)ctx->num_sms * 8);
  if (from == FTN_F64 && to == FTN_F32)
    cast_batch_kernel<double, float><<<g, 256, 0, ctx->stream>>>(d_jobs, njobs, tiles);
  else if (from == FTN_F32 && to == FTN_F64)
    cast_batch_kernel<float, double><<<g, 256, 0, ctx->stream>>>(d_jobs, njobs, tiles);
  else if (from == FTN_F64)
    cast_batch_kernel<double, double><<<g, 256, 0, ctx->stream>>>(d_jobs, njobs, tiles);
  else
    cast_batch_kernel<float, float><<<g, 256, 0, ctx->stream>>>(d_jobs, njobs, tiles);
  ctx->launches += 1;
  FTN_CUDA(cudaGetLastError());
  return FTN_OK;
}

__global__ void gather_results_kernel(const ResultJob* __restrict__ jobs, int njobs, double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < njobs; i += gridDim.x * blockDim.x) {
    const ResultJob J = jobs[i];
    double v = 0.0;
    if (J.value) v = J.f64 ? *reinterpret_cast<const double*>(J.value) : (double)*reinterpret_cast<const float*>(J.value);
    out[2 * i] = J.sign < 0 ? -v : v;
    out[2 * i + 1] = *J.logacc;
  }
}

ftn_status launch_gather_results(ftn_ctx ctx, const ResultJob* d_jobs, int njobs, double* out) {
  if (njobs == 0) return FTN_OK;
  gather_results_kernel<<<(unsigned)((njobs + 255) / 256), 256, 0, ctx->stream>>>(d_jobs, njobs, out);
  ctx->launches += 1;
  FTN_CUDA(cudaGetLastError());
  return FTN_OK;
}

// One thread waits on an mbarrier phase that nothing completes, through the
// same bounded-wait helper the tensor-core GEMM and the staged permute use,
// so the wait gives up after limit_ns, records DEV_ERR_TIMEOUT in the error
// word and the kernel returns.
__global__ void wait_selftest_kernel(int* err, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  mbar_init(&bar, 1);
  fence_mbar_init();
  mbar_wait_for(&bar, 0, err, limit_ns, false);
}

ftn_status launch_wait_selftest(ftn_ctx ctx, uint64_t limit_ns) {
  wait_selftest_kernel<<<1, 1, 0, ctx->stream>>>(ctx->dev_err, limit_ns);
  ctx->launches += 1;
  FTN_CUDA(cudaGetLastError());
  return FTN_OK;
}

}  // namespace ftn
