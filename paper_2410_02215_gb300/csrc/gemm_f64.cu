// Grouped FP64 sector GEMM (plain FP64 path): C[m, n] = sum_k A[m, k] B[n, k]
// for every (row block, column block) pair of a fermionic contraction, both
// operands K-major in the fused sector-matrix layout.  tcgen05 has no FP64
// kind, so these are DFMA kernels: 64 x bn tiles with 4 x (bn / 16) outputs
// per thread over a persistent grid for problems of more than 4096 outputs,
// one warp per group of outputs for the smaller ones.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "common.h"
#include "ptx.cuh"

namespace ftn {

constexpr int F64_BM = 64, F64_BK = 16;

__device__ __forceinline__ int find_prob(const GemmProb* probs, int nprobs, int64_t t) {
  int lo = 0, hi = nprobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile_begin <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// 64 x BN tiles (BN = 16, 32 or 64, chosen per launch from the widest
// problem): 256 threads, 4 x (BN / 16) outputs each.  FP64 is the bound, so
// the tile width follows the problems' column counts instead of wasting
// DFMAs on padding columns.
template <int BN>
__global__ void __launch_bounds__(256) gemm_f64_kernel(const GemmProb* __restrict__ probs, int nprobs, int64_t tiles,
                                                       const double* __restrict__ A, const double* __restrict__ B,
                                                       double* __restrict__ C) {
  constexpr int TN = BN / 16;
  __shared__ double As[F64_BK][F64_BM + 1];
  __shared__ double Bs[F64_BK][BN + 1];
  __shared__ int s_p;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    if (tid == 0) s_p = find_prob(probs, nprobs, t);
    __syncthreads();
    const GemmProb& p = probs[s_p];
    int64_t local = t - p.tile_begin;
    const int nsp = p.nsplit > 1 ? p.nsplit : 1;
    const int ks = (int)(local % nsp);
    local /= nsp;
    const int m0 = (int)(local / p.tiles_n) * F64_BM;
    const int n0 = (int)(local % p.tiles_n) * BN;
    const int kbeg = nsp > 1 ? ks * p.kchunk : 0;
    const int kend = nsp > 1 ? min(p.K, kbeg + p.kchunk) : p.K;
    double acc[4][TN];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < TN; ++c) acc[a][c] = 0.0;
    const double* Ap = A + p.a_off;
    const double* Bp = B + p.b_off;
    const bool a_kfast = p.a_sk == 1, b_kfast = p.b_sk == 1;
    for (int k0 = kbeg; k0 < kend; k0 += F64_BK) {
      // threads run along whichever operand index has unit stride
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int idx = tid + 256 * e;
        const int row = a_kfast ? idx >> 4 : idx & 63, kk = a_kfast ? idx & 15 : idx >> 6;
        const int gm = m0 + row, gk = k0 + kk;
        As[kk][row] = (gm < p.M && gk < kend) ? Ap[(int64_t)gm * p.a_sm + (int64_t)gk * p.a_sk] : 0.0;
      }
#pragma unroll
      for (int e = 0; e < TN; ++e) {
        const int idx = tid + 256 * e;
        const int row = b_kfast ? idx >> 4 : idx % BN, kk = b_kfast ? idx & 15 : idx / BN;
        const int gn = n0 + row, gk = k0 + kk;
        Bs[kk][row] = (gn < p.N && gk < kend) ? Bp[(int64_t)gn * p.b_sn + (int64_t)gk * p.b_sk] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < F64_BK; ++kk) {
        double av[4], bv[TN];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
        for (int c = 0; c < TN; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < TN; ++c) acc[a][c] = fma(av[a], bv[c], acc[a][c]);
      }
      __syncthreads();
    }
    int64_t cpart[TN];
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      int gn = n0 + tx + 16 * c;
      cpart[c] = gn < p.N ? expand_index32(gn, p.ncl, p.cdim, p.cstr) : 0;
    }
    const double sg = (double)p.c_sign;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int gm = m0 + ty + 16 * a;
      if (gm >= p.M) continue;
      const int64_t rpart = p.c_off + (int64_t)ks * p.c_slab + expand_index32(gm, p.nrl, p.rdim, p.rstr);
#pragma unroll
      for (int c = 0; c < TN; ++c) {
        int gn = n0 + tx + 16 * c;
        if (gn < p.N) C[rpart + cpart[c]] = sg * acc[a][c];
      }
    }
    __syncthreads();
  }
}

int f64_pick_bn(int max_n) { return max_n <= 16 ? 16 : max_n <= 32 ? 32 : 64; }

// Small problems: one warp per item of up to F64W_PASSES passes.  Pass q
// gives each group of g lanes one output (m, n) = (e / N, e % N); the item's
// passes run together, so the loads of all its outputs are in flight at once
// (the operands come straight from global memory, L1-cached: latency, not
// bandwidth or FP64 rate, bounds these short dot products).  Lane kl of a
// group sums the terms k = kl, kl + g, ... of its split slice in order, and
// the group's partial sums are added by a butterfly over the g lanes.
__global__ void __launch_bounds__(128, 6) gemm_f64_warp_kernel(const GemmProb* __restrict__ probs,
                                                               const WarpItem* __restrict__ items, int nitems,
                                                               const double* __restrict__ A,
                                                               const double* __restrict__ B, double* __restrict__ C) {
  constexpr int P = F64W_PASSES;
  const int lane = threadIdx.x & 31;
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); w < nitems; w += nw) {
    const WarpItem it = items[w];
    const GemmProb* __restrict__ p = probs + it.prob;
    const int N = p->N, K = p->K;
    const int nsp = p->nsplit > 1 ? p->nsplit : 1;
    const int kbeg = nsp > 1 ? it.ks * p->kchunk : 0;
    const int kend = nsp > 1 ? min(K, kbeg + p->kchunk) : K;
    const int g = f64w_klanes(nsp > 1 ? p->kchunk : K);
    const int lg = __ffs(g) - 1, opp = 32 >> lg;
    const int o = lane >> lg, kl = lane & (g - 1);
    const int64_t a_sm = p->a_sm, a_sk = p->a_sk, b_sn = p->b_sn, b_sk = p->b_sk;
    const double* ar[P];
    const double* br[P];
    bool vq[P];
    double s[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int le = q * opp + o;
      vq[q] = le < it.cnt;
      const int e = it.e0 + (vq[q] ? le : 0);
      const int m = e / N;
      ar[q] = A + p->a_off + (int64_t)m * a_sm;
      br[q] = B + p->b_off + (int64_t)(e - m * N) * b_sn;
      s[q] = 0.0;
    }
    for (int k = kbeg + kl; k < kend; k += g) {
#pragma unroll
      for (int q = 0; q < P; ++q)
        if (vq[q]) s[q] = fma(ar[q][(int64_t)k * a_sk], br[q][(int64_t)k * b_sk], s[q]);
    }
    const int64_t cbase = p->c_off + (int64_t)it.ks * p->c_slab;
    const double sg = (double)p->c_sign;
#pragma unroll
    for (int q = 0; q < P; ++q) {
      double acc = s[q];
      for (int off = 1; off < g; off <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (vq[q] && kl == 0) {
        const int e = it.e0 + q * opp + o, m = e / N;
        C[cbase + expand_index32(m, p->nrl, p->rdim, p->rstr) + expand_index32(e - m * N, p->ncl, p->cdim, p->cstr)] =
            sg * acc;
      }
    }
  }
}

// Small tensor-core-precision problems (the same size bound) on CUDA cores:
// each operand element is its stored planes added in FP32 (hi + lo for the
// split precisions, hi alone otherwise), products accumulated in FP32 FMAs.
// That is at least as accurate as the tensor-core passes of the precision,
// which multiply the same planes; the lane, pass and butterfly structure is
// the FP64 warp kernel's.
template <typename T>
__device__ __forceinline__ float plane_val(const T* p) {
  if constexpr (sizeof(T) == 4)
    return *reinterpret_cast<const float*>(p);
  else if constexpr (std::is_same<T, __half>::value)
    return __half2float(*p);
  else
    return __bfloat162float(*p);
}

template <typename T, bool SPLIT>
__global__ void __launch_bounds__(128, 8) gemm_f32_warp_kernel(const GemmProb* __restrict__ probs,
                                                               const WarpItem* __restrict__ items, int nitems,
                                                               const T* __restrict__ A, const T* __restrict__ B,
                                                               int64_t lo_delta, float* __restrict__ C) {
  constexpr int P = F64W_PASSES;
  const int lane = threadIdx.x & 31;
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); w < nitems; w += nw) {
    const WarpItem it = items[w];
    const GemmProb* __restrict__ p = probs + it.prob;
    const int N = p->N, K = p->K;
    const int g = f64w_klanes(K);
    const int lg = __ffs(g) - 1, opp = 32 >> lg;
    const int o = lane >> lg, kl = lane & (g - 1);
    const int64_t a_sm = p->a_sm, a_sk = p->a_sk, b_sn = p->b_sn, b_sk = p->b_sk;
    const T* ar[P];
    const T* br[P];
    bool vq[P];
    float s[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int le = q * opp + o;
      vq[q] = le < it.cnt;
      const int e = it.e0 + (vq[q] ? le : 0);
      const int m = e / N;
      ar[q] = A + p->a_off + (int64_t)m * a_sm;
      br[q] = B + p->b_off + (int64_t)(e - m * N) * b_sn;
      s[q] = 0.0f;
    }
    for (int k = kl; k < K; k += g) {
#pragma unroll
      for (int q = 0; q < P; ++q)
        if (vq[q]) {
          const T* pa = ar[q] + (int64_t)k * a_sk;
          const T* pb = br[q] + (int64_t)k * b_sk;
          float a = plane_val(pa), b = plane_val(pb);
          if constexpr (SPLIT) {
            a += plane_val(pa + lo_delta);
            b += plane_val(pb + lo_delta);
          }
          s[q] = fmaf(a, b, s[q]);
        }
    }
    const float sg = (float)p->c_sign;
#pragma unroll
    for (int q = 0; q < P; ++q) {
      float acc = s[q];
      for (int off = 1; off < g; off <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (vq[q] && kl == 0) {
        const int e = it.e0 + q * opp + o, m = e / N;
        C[p->c_off + expand_index32(m, p->nrl, p->rdim, p->rstr) + expand_index32(e - m * N, p->ncl, p->cdim, p->cstr)] =
            sg * acc;
      }
    }
  }
}

ftn_status launch_gemm_f32_warp(ftn_ctx ctx, ftn_prec prec, const GemmProb* d_probs, const WarpItem* d_items,
                                int nitems, const void* a, const void* b, int64_t lo_delta, float* c) {
  if (nitems == 0) return FTN_OK;
  int64_t grid = ((int64_t)nitems + 3) / 4;
  const int64_t cap = (int64_t)ctx->num_sms * 8;
  if (grid > cap) grid = cap;
  const unsigned gd = (unsigned)grid;
  cudaStream_t s = ctx->stream;
  switch (prec) {
    case FTN_PREC_TF32:
      gemm_f32_warp_kernel<float, false><<<gd, 128, 0, s>>>(d_probs, d_items, nitems, (const float*)a,
                                                            (const float*)b, lo_delta, c);
      break;
    case FTN_PREC_TF32X3:
      gemm_f32_warp_kernel<float, true><<<gd, 128, 0, s>>>(d_probs, d_items, nitems, (const float*)a,
                                                           (const float*)b, lo_delta, c);
      break;
    case FTN_PREC_BF16:
      gemm_f32_warp_kernel<__nv_bfloat16, false><<<gd, 128, 0, s>>>(
          d_probs, d_items, nitems, (const __nv_bfloat16*)a, (const __nv_bfloat16*)b, lo_delta, c);
      break;
    case FTN_PREC_BF16X3:
      gemm_f32_warp_kernel<__nv_bfloat16, true><<<gd, 128, 0, s>>>(
          d_probs, d_items, nitems, (const __nv_bfloat16*)a, (const __nv_bfloat16*)b, lo_delta, c);
      break;
    case FTN_PREC_F16X3:
      gemm_f32_warp_kernel<__half, true><<<gd, 128, 0, s>>>(d_probs, d_items, nitems, (const __half*)a,
                                                            (const __half*)b, lo_delta, c);
      break;
    default:
      return set_error(FTN_EINVAL, "internal error: CUDA-core GEMM precision");
  }
  ctx->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "gemm_f32_warp_kernel launch");
  return FTN_OK;
}

void f64w_items(const GemmProb& g, int prob, std::vector<WarpItem>& out) {
  const int nsp = g.nsplit > 1 ? g.nsplit : 1;
  const int per = (32 / f64w_klanes(nsp > 1 ? g.kchunk : g.K)) * F64W_PASSES;
  const int64_t mn = (int64_t)g.M * g.N;
  for (int s = 0; s < nsp; ++s)
    for (int64_t e = 0; e < mn; e += per) out.push_back({prob, s, (int32_t)e, (int32_t)std::min<int64_t>(per, mn - e)});
}

int partition_f64(std::vector<GemmProb>& probs, std::vector<WarpItem>& items, int64_t& tiles) {
  std::stable_partition(probs.begin(), probs.end(), [](const GemmProb& g) { return !f64w_small(g); });
  items.clear();
  tiles = 0;
  int nt = 0;
  for (size_t i = 0; i < probs.size(); ++i) {
    GemmProb& g = probs[i];
    if (f64w_small(g)) {
      f64w_items(g, (int)i, items);
      continue;
    }
    g.tile_begin = tiles;
    tiles += (int64_t)g.tiles_m * g.tiles_n * (g.nsplit > 1 ? g.nsplit : 1);
    ++nt;
  }
  return nt;
}

ftn_status launch_gemm_f64_warp(ftn_ctx ctx, const GemmProb* d_probs, const WarpItem* d_items, int nitems,
                                const double* a, const double* b, double* c) {
  if (nitems == 0) return FTN_OK;
  int64_t grid = ((int64_t)nitems + 3) / 4;
  const int64_t cap = (int64_t)ctx->num_sms * 6;  // resident CTAs (at most 80 registers, 128 threads)
  if (grid > cap) grid = cap;
  gemm_f64_warp_kernel<<<(unsigned)grid, 128, 0, ctx->stream>>>(d_probs, d_items, nitems, a, b, c);
  ctx->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "gemm_f64_warp_kernel launch");
  return FTN_OK;
}

__global__ void sum_slabs_kernel(double* __restrict__ dst, const double* __restrict__ src, int64_t count, int nsplit,
                                 int64_t slab) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < nsplit; ++s) acc += src[s * slab + e];
    dst[e] = acc;
  }
}

ftn_status launch_sum_slabs(ftn_ctx ctx, double* dst, const double* src, int64_t count, int nsplit, int64_t slab) {
  if (count <= 0) return FTN_OK;
  int64_t grid = (count + 255) / 256;
  if (grid > (int64_t)ctx->num_sms * 8) grid = (int64_t)ctx->num_sms * 8;
  sum_slabs_kernel<<<(unsigned)grid, 256, 0, ctx->stream>>>(dst, src, count, nsplit, slab);
  ctx->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "sum_slabs_kernel launch");
  return FTN_OK;
}

// Split-K reduction with the problems' own epilogues: red[i] carries the
// epilogue mapping of problem i (c_off, row/column leg dims and strides,
// sign), a_off = its partial slabs' offset in `part`, nsplit slabs of
// c_slab = M * N elements, and tile_begin = its first element in the
// flattened element list.  Slabs are added in split order, so the result
// does not depend on the launch.
__global__ void splitk_reduce_kernel(const GemmProb* __restrict__ red, int nred, int64_t total,
                                     const double* __restrict__ part, double* __restrict__ C) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const GemmProb& g = red[find_prob(red, nred, e)];
    const int64_t local = e - g.tile_begin;
    const int m = (int)(local / g.N), n = (int)(local - (int64_t)m * g.N);
    const double* src = part + g.a_off + local;
    double acc = 0.0;
    for (int s = 0; s < g.nsplit; ++s) acc += src[(int64_t)s * g.c_slab];
    C[g.c_off + expand_index32(m, g.nrl, g.rdim, g.rstr) + expand_index32(n, g.ncl, g.cdim, g.cstr)] =
        (double)g.c_sign * acc;
  }
}

// FP32 partial slabs (tensor-core K-split parts), added in FP64.
__global__ void splitk_reduce_f32_kernel(const GemmProb* __restrict__ red, int nred, int64_t total,
                                         const float* __restrict__ part, float* __restrict__ C) {
  // launched with programmatic serialisation (the adjoint's reduction follows its GEMM on one
  // stream): nothing is read before this
  pdl_wait();
  pdl_launch_dependents();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const GemmProb& g = red[find_prob(red, nred, e)];
    const int64_t local = e - g.tile_begin;
    const int m = (int)(local / g.N), n = (int)(local - (int64_t)m * g.N);
    const float* src = part + g.a_off + local;
    double acc = 0.0;
    for (int s = 0; s < g.nsplit; ++s) acc += (double)src[(int64_t)s * g.c_slab];
    C[g.c_off + expand_index32(m, g.nrl, g.rdim, g.rstr) + expand_index32(n, g.ncl, g.cdim, g.cstr)] =
        (float)((double)g.c_sign * acc);
  }
}

ftn_status launch_splitk_reduce_f32(ftn_ctx ctx, const GemmProb* d_red, int nred, int64_t total, const float* part,
                                    float* c) {
  if (nred == 0 || total == 0) return FTN_OK;
  int64_t grid = (total + 255) / 256;
  if (grid > (int64_t)ctx->num_sms * 8) grid = (int64_t)ctx->num_sms * 8;
  launch_pdl(splitk_reduce_f32_kernel, (unsigned)grid, 256, 0, ctx->stream, d_red, nred, total, part, c);
  ctx->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "splitk_reduce_f32_kernel launch");
  return FTN_OK;
}

int64_t plan_splitk_f64(std::vector<GemmProb>& probs, int num_sms, std::vector<GemmProb>& red, int64_t& tiles,
                        int64_t& red_total) {
  red.clear();
  red_total = 0;
  int64_t t0 = 0;
  int kmax = 0;
  for (const GemmProb& g : probs) {
    t0 += (int64_t)g.tiles_m * g.tiles_n;
    kmax = std::max(kmax, g.K);
  }
  if (probs.empty() || t0 >= 2 * (int64_t)num_sms || kmax < 64) return 0;
  const int64_t want = (2 * (int64_t)num_sms + t0 - 1) / t0;
  int64_t part = 0, elems = 0, tb = 0;
  for (GemmProb& g : probs) {
    GemmProb r = g;  // keeps the epilogue
    int s = (int)std::min<int64_t>(std::min<int64_t>(want, 64), std::max(1, (g.K + 15) / 16));
    int kchunk = std::max(16, ((g.K + s - 1) / s + 15) / 16 * 16);
    s = std::max(1, (g.K + kchunk - 1) / kchunk);
    const int64_t mn = (int64_t)g.M * g.N;
    r.a_off = part;
    r.nsplit = s;
    r.c_slab = mn;
    r.tile_begin = elems;
    red.push_back(r);
    g.nsplit = s;
    g.kchunk = kchunk;
    gemm_plain_output(g, part, g.N);
    g.c_slab = mn;
    g.tile_begin = tb;
    tb += (int64_t)g.tiles_m * g.tiles_n * s;
    part += mn * s;
    elems += mn;
  }
  tiles = tb;
  red_total = elems;
  return part;
}

bool red_in_bounds(const std::vector<GemmProb>& red, int64_t part_n, int64_t c_n) {
  for (const GemmProb& g : red) {
    if (g.M <= 0 || g.N <= 0 || g.nsplit < 1 || g.c_slab != (int64_t)g.M * g.N) return false;
    if (g.a_off < 0 || g.a_off + (int64_t)g.nsplit * g.c_slab > part_n) return false;
    int64_t mr = 1, mc = 1, top = g.c_off;
    for (int l = 0; l < g.nrl; ++l) mr *= g.rdim[l], top += (int64_t)(g.rdim[l] - 1) * g.rstr[l];
    for (int l = 0; l < g.ncl; ++l) mc *= g.cdim[l], top += (int64_t)(g.cdim[l] - 1) * g.cstr[l];
    if (mr != g.M || mc != g.N || g.c_off < 0 || top >= c_n) return false;
  }
  return true;
}

ftn_status launch_splitk_reduce(ftn_ctx ctx, const GemmProb* d_red, int nred, int64_t total, const double* part,
                                double* c) {
  if (nred == 0 || total == 0) return FTN_OK;
  int64_t grid = (total + 255) / 256;
  if (grid > (int64_t)ctx->num_sms * 8) grid = (int64_t)ctx->num_sms * 8;
  splitk_reduce_kernel<<<(unsigned)grid, 256, 0, ctx->stream>>>(d_red, nred, total, part, c);
  ctx->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "splitk_reduce_kernel launch");
  return FTN_OK;
}

void gemm_plain_output(GemmProb& g, int64_t c_off, int64_t ld) {
  g.c_off = c_off;
  g.c_sign = 1;
  g.nrl = g.ncl = 1;
  g.rdim[0] = g.M;
  g.rstr[0] = ld;
  g.cdim[0] = g.N;
  g.cstr[0] = 1;
}

ftn_status launch_gemm_f64(ftn_ctx ctx, const GemmProb* d_probs, int nprobs, int64_t tiles, const double* a,
                           const double* b, double* c, int bn) {
  if (nprobs == 0 || tiles == 0) return FTN_OK;
  int64_t grid = tiles;
  int64_t cap = (int64_t)ctx->num_sms * 4;
  if (grid > cap) grid = cap;
  if (bn == 16)
    gemm_f64_kernel<16><<<(unsigned)grid, 256, 0, ctx->stream>>>(d_probs, nprobs, tiles, a, b, c);
  else if (bn == 32)
    gemm_f64_kernel<32><<<(unsigned)grid, 256, 0, ctx->stream>>>(d_probs, nprobs, tiles, a, b, c);
  else if (bn == 64)
    gemm_f64_kernel<64><<<(unsigned)grid, 256, 0, ctx->stream>>>(d_probs, nprobs, tiles, a, b, c);
  else
    return set_error(FTN_EINVAL, "internal error: FP64 GEMM tile width");
  ctx->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "gemm_f64_kernel launch");
  return FTN_OK;
}

}  // namespace ftn
