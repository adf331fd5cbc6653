// Sign-permute kernel: moves every block of a graded tensor into a new leg
// order or into the fused sector-matrix layout of a contraction, multiplying
// it by its fermionic sign (one sign per block: every factor of Eq.
// (transposition), of the bond parity g and of the fusion order depends only
// on the block's parity bits).
//
// Each CTA tile covers PERM_TO rows of the O group (destination-fast legs)
// times PERM_TI elements of the I group (the source's contiguous suffix) for
// one batch index.  Loads run along I (coalesced in the source); stores run
// along O through a shared-memory transpose, or directly along I when the
// destination is also contiguous there.  Every thread keeps PERM_TO / 8 loads
// in flight so that enough bytes are outstanding per SM to cover HBM latency.
#include <cuda_bf16.h>

#include "common.h"

namespace ftn {

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

template <typename Tin, int MODE>
__device__ __forceinline__ void put(void* dst0, void* dst1, int64_t idx, Tin v) {
  if constexpr (MODE == PERM_SAME) {
    reinterpret_cast<Tin*>(dst0)[idx] = v;
  } else if constexpr (MODE == PERM_TF32) {
    reinterpret_cast<float*>(dst0)[idx] = tf32_rna((float)v);
  } else if constexpr (MODE == PERM_TF32X2) {
    float hi = tf32_rna((float)v);
    reinterpret_cast<float*>(dst0)[idx] = hi;
    reinterpret_cast<float*>(dst1)[idx] = tf32_rna((float)v - hi);
  } else if constexpr (MODE == PERM_BF16) {
    reinterpret_cast<__nv_bfloat16*>(dst0)[idx] = __float2bfloat16_rn((float)v);
  } else {
    __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
    reinterpret_cast<__nv_bfloat16*>(dst0)[idx] = hi;
    reinterpret_cast<__nv_bfloat16*>(dst1)[idx] = __float2bfloat16_rn((float)v - __bfloat162float(hi));
  }
}

constexpr int PT = 256;              // threads per CTA
constexpr int PR = PERM_TO / (PT / 32);  // rows per thread in a phase

template <typename Tin, int MODE>
__global__ void __launch_bounds__(PT) perm_kernel(const PermJob* __restrict__ jobs, int njobs, int64_t tiles,
                                                  const Tin* __restrict__ src, void* __restrict__ dst0,
                                                  void* __restrict__ dst1) {
  __shared__ Tin tile[PERM_TO][PERM_TI + 1];
  __shared__ int32_t rowS[PERM_TO];
  __shared__ int32_t rowD[PERM_TO];
  __shared__ int32_t colD[PERM_TI];
  __shared__ int64_t baseS, baseD;
  __shared__ int s_job;
  const int tid = threadIdx.x;
  const int tx = tid & 31, ty = tid >> 5;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    if (tid == 0) {
      int lo = 0, hi = njobs - 1;
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].tile_begin <= t)
          lo = mid;
        else
          hi = mid - 1;
      }
      s_job = lo;
    }
    __syncthreads();
    const PermJob* j = jobs + s_job;
    const int nI = j->nI, nO = j->nO;
    const int PI = j->PI, PO = j->PO;
    const int64_t local = t - j->tile_begin;
    const int64_t per_b = (int64_t)j->tiles_i * j->tiles_o;
    const int64_t b = local / per_b;
    const int rem = (int)(local - b * per_b);
    const int ti = rem % j->tiles_i, to = rem / j->tiles_i;
    if (tid == PT - 1) {
      int64_t s = j->src_off, d = j->dst_off, x = b;
      for (int q = nI + nO + j->nB - 1; q >= nI + nO; --q) {
        int64_t idx = x % j->dim[q];
        x /= j->dim[q];
        s += idx * j->sstr[q];
        d += idx * j->dstr[q];
      }
      baseS = s;
      baseD = d;
    }
    if (tid < PERM_TO) {
      int o = to * PERM_TO + tid;
      int32_t s = 0, d = 0;
      if (o < PO) {
        int x = o;
        for (int q = nI + nO - 1; q >= nI; --q) {
          int idx = x % j->dim[q];
          x /= j->dim[q];
          s += idx * (int32_t)j->sstr[q];
          d += idx * (int32_t)j->dstr[q];
        }
      }
      rowS[tid] = s;
      rowD[tid] = d;
    } else if (tid < PERM_TO + PERM_TI) {
      int c = tid - PERM_TO;
      int i = ti * PERM_TI + c;
      int32_t d = 0;
      if (i < PI) {
        int x = i;
        for (int q = nI - 1; q >= 0; --q) {
          int idx = x % j->dim[q];
          x /= j->dim[q];
          d += idx * (int32_t)j->dstr[q];
        }
      }
      colD[c] = d;
    }
    __syncthreads();
    const int i = ti * PERM_TI + tx;
    const Tin sgn = (Tin)j->sign;
    const int64_t bS = baseS, bD = baseD;
    const int o0 = to * PERM_TO;
    if (j->store_fast_i) {
      // destination contiguous along I: copy straight through registers
      Tin v[PR];
#pragma unroll
      for (int r = 0; r < PR; ++r) {
        int row = ty + r * (PT / 32);
        v[r] = (o0 + row < PO && i < PI) ? src[bS + rowS[row] + i] : Tin(0);
      }
      const int32_t cd = colD[tx];
#pragma unroll
      for (int r = 0; r < PR; ++r) {
        int row = ty + r * (PT / 32);
        if (o0 + row < PO && i < PI) put<Tin, MODE>(dst0, dst1, bD + rowD[row] + cd, sgn * v[r]);
      }
    } else {
#pragma unroll
      for (int r = 0; r < PR; ++r) {
        int row = ty + r * (PT / 32);
        if (o0 + row < PO && i < PI) tile[row][tx] = src[bS + rowS[row] + i];
      }
      __syncthreads();
      // stores along O: lane -> row, warps -> columns of I
#pragma unroll
      for (int half = 0; half < PERM_TO / 32; ++half) {
        const int row = half * 32 + tx;
        const bool okr = o0 + row < PO;
        const int32_t rd = rowD[row];
#pragma unroll
        for (int c = ty; c < PERM_TI; c += PT / 32) {
          const int i2 = ti * PERM_TI + c;
          if (okr && i2 < PI) put<Tin, MODE>(dst0, dst1, bD + rd + colD[c], sgn * tile[row][c]);
        }
      }
    }
    __syncthreads();
  }
}

template <typename Tin, int MODE>
static cudaError_t go(ftn_ctx ctx, const PermJob* d_jobs, int njobs, int64_t tiles, const void* src, void* dst0,
                      void* dst1) {
  int64_t grid = tiles;
  int64_t cap = (int64_t)ctx->num_sms * 16;
  if (grid > cap) grid = cap;
  perm_kernel<Tin, MODE><<<(unsigned)grid, PT, 0, ctx->stream>>>(d_jobs, njobs, tiles, (const Tin*)src, dst0, dst1);
  return cudaGetLastError();
}

ftn_status launch_permute(ftn_ctx ctx, const PermJob* d_jobs, int njobs, int64_t tiles, const void* src, void* dst0,
                          void* dst1, ftn_dtype in_type, int mode) {
  if (njobs == 0 || tiles == 0) return FTN_OK;
  cudaError_t e;
  if (in_type == FTN_F64) {
    if (mode != PERM_SAME) return set_error(FTN_EUNSUPPORTED, "FP64 permute supports only the same-type output");
    e = go<double, PERM_SAME>(ctx, d_jobs, njobs, tiles, src, dst0, dst1);
  } else {
    switch (mode) {
      case PERM_SAME: e = go<float, PERM_SAME>(ctx, d_jobs, njobs, tiles, src, dst0, dst1); break;
      case PERM_TF32: e = go<float, PERM_TF32>(ctx, d_jobs, njobs, tiles, src, dst0, dst1); break;
      case PERM_TF32X2: e = go<float, PERM_TF32X2>(ctx, d_jobs, njobs, tiles, src, dst0, dst1); break;
      case PERM_BF16: e = go<float, PERM_BF16>(ctx, d_jobs, njobs, tiles, src, dst0, dst1); break;
      case PERM_BF16X2: e = go<float, PERM_BF16X2>(ctx, d_jobs, njobs, tiles, src, dst0, dst1); break;
      default: return set_error(FTN_EINVAL, "bad permute mode");
    }
  }
  ctx->launches += 1;
  if (e != cudaSuccess) return cuda_error(e, "perm_kernel launch");
  return FTN_OK;
}

}  // namespace ftn
