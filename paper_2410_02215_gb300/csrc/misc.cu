// Small device kernels used by the contraction-tree executor: per-step
// max-abs normalisation with an FP64 log-scale accumulator kept on the
// device (no host round trip), and FP32 <-> FP64 casts.
#include "common.h"

namespace ftn {

// d_state[0]: running max |x| of the current tensor (as ordered bits of a
// non-negative double); d_state[1]: log-scale accumulator (double).
template <typename T>
__global__ void maxabs_kernel(const T* __restrict__ x, int64_t n, unsigned long long* __restrict__ mx) {
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs((double)x[i]));
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(mx, (unsigned long long)__double_as_longlong(m));
}

template <typename T>
__global__ void scale_kernel(T* __restrict__ x, int64_t n, const unsigned long long* __restrict__ mx,
                             double* __restrict__ logacc) {
  const double m = __longlong_as_double((long long)*mx);
  if (!(m > 0.0)) return;
  const T inv = (T)(1.0 / m);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) *logacc += log(m);
}

template <typename Ti, typename To>
__global__ void cast_kernel(const Ti* __restrict__ x, To* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (To)x[i];
}

static unsigned grid_for(ftn_ctx ctx, int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > (int64_t)ctx->num_sms * 8) g = (int64_t)ctx->num_sms * 8;
  return (unsigned)(g < 1 ? 1 : g);
}

ftn_status normalize_tensor(ftn_ctx ctx, ftn_tensor t, void* d_state) {
  unsigned long long* mx = (unsigned long long*)d_state;
  double* logacc = (double*)((char*)d_state + 8);
  FTN_CUDA(cudaMemsetAsync(mx, 0, 8, ctx->stream));
  if (t->numel == 0) return FTN_OK;
  const unsigned g = grid_for(ctx, t->numel);
  if (t->dtype == FTN_F64) {
    maxabs_kernel<double><<<g, 256, 0, ctx->stream>>>((const double*)t->data, t->numel, mx);
    scale_kernel<double><<<g, 256, 0, ctx->stream>>>((double*)t->data, t->numel, mx, logacc);
  } else {
    maxabs_kernel<float><<<g, 256, 0, ctx->stream>>>((const float*)t->data, t->numel, mx);
    scale_kernel<float><<<g, 256, 0, ctx->stream>>>((float*)t->data, t->numel, mx, logacc);
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

}  // namespace ftn
