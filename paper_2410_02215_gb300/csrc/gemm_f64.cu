// Grouped FP64 sector GEMM (plain FP64 path): C[m, n] = sum_k A[m, k] B[n, k]
// for every (row block, column block) pair of a fermionic contraction, both
// operands K-major in the fused sector-matrix layout.  tcgen05 has no FP64
// kind, so this is a DFMA kernel: 64x64 tiles, 4x4 outputs per thread,
// persistent grid over the flattened tile list of all problems.
#include "common.h"

namespace ftn {

constexpr int F64_BM = 64, F64_BN = 64, F64_BK = 16;

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

__global__ void __launch_bounds__(256) gemm_f64_kernel(const GemmProb* __restrict__ probs, int nprobs, int64_t tiles,
                                                       const double* __restrict__ A, const double* __restrict__ B,
                                                       double* __restrict__ C) {
  __shared__ double As[F64_BK][F64_BM + 1];
  __shared__ double Bs[F64_BK][F64_BN + 1];
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
    const int n0 = (int)(local % p.tiles_n) * F64_BN;
    const int kbeg = nsp > 1 ? ks * p.kchunk : 0;
    const int kend = nsp > 1 ? min(p.K, kbeg + p.kchunk) : p.K;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c] = 0.0;
    const double* Ap = A + p.a_off;
    const double* Bp = B + p.b_off;
    const bool a_kfast = p.a_sk == 1, b_kfast = p.b_sk == 1;
    for (int k0 = kbeg; k0 < kend; k0 += F64_BK) {
      // threads run along whichever operand index has unit stride
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        int idx = tid + 256 * e;
        int row = a_kfast ? idx >> 4 : idx & 63, kk = a_kfast ? idx & 15 : idx >> 6;
        int gm = m0 + row, gk = k0 + kk;
        As[kk][row] = (gm < p.M && gk < kend) ? Ap[(int64_t)gm * p.a_sm + (int64_t)gk * p.a_sk] : 0.0;
        row = b_kfast ? idx >> 4 : idx & 63;
        kk = b_kfast ? idx & 15 : idx >> 6;
        gk = k0 + kk;
        int gn = n0 + row;
        Bs[kk][row] = (gn < p.N && gk < kend) ? Bp[(int64_t)gn * p.b_sn + (int64_t)gk * p.b_sk] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < F64_BK; ++kk) {
        double av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
        for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a][c] = fma(av[a], bv[c], acc[a][c]);
      }
      __syncthreads();
    }
    int64_t cpart[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
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
      for (int c = 0; c < 4; ++c) {
        int gn = n0 + tx + 16 * c;
        if (gn < p.N) C[rpart + cpart[c]] = sg * acc[a][c];
      }
    }
    __syncthreads();
  }
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
                           const double* b, double* c) {
  if (nprobs == 0 || tiles == 0) return FTN_OK;
  int64_t grid = tiles;
  int64_t cap = (int64_t)ctx->num_sms * 4;
  if (grid > cap) grid = cap;
  gemm_f64_kernel<<<(unsigned)grid, 256, 0, ctx->stream>>>(d_probs, nprobs, tiles, a, b, c);
  ctx->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "gemm_f64_kernel launch");
  return FTN_OK;
}

}  // namespace ftn
