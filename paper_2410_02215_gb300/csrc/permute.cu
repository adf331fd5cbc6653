// Sign-permute kernel: moves every block of a graded tensor into a new leg
// order or into the fused sector-matrix layout of a contraction, multiplying
// it by its fermionic sign (one sign per block: every factor of Eq.
// (transposition), of the bond parity g and of the fusion order depends only
// on the block's parity bits).
//
// Two kernels share the job format.  The staged kernel (used when every
// source row of a job starts 16-byte aligned): each persistent CTA takes a
// contiguous range of tiles; two producer warps (alternate tiles) build a
// tile's row and column tables -- with the job and multiply-shift
// reciprocals of its leg dimensions cached in shared memory -- and copy its
// source rows into a PERM_STAGES-deep shared-memory ring with 16-byte
// cp.async copies spread over their lanes (consecutive lanes on consecutive
// chunks of a row; completion tracked on an mbarrier), while six writer
// warps write earlier tiles out along the destination's contiguous direction,
// releasing ring slots through a second set of mbarriers (no block-wide
// synchronisation in the loop).  The copies hold no registers while in
// flight.  (One bulk copy per row was tried first: a few hundred cycles per
// request per SM left the rows of 128 to 512 bytes far below the HBM
// bandwidth.  All warps building tables and copying between block barriers
// was tried next: the tables then ran in series with the writes.)  The
// fallback kernel stages through registers:
// Each CTA tile covers PERM_TO rows of the O group (destination-fast legs)
// times PERM_TI elements of the I group (the source's contiguous suffix) for
// one batch index.  Loads run along I (coalesced in the source); stores run
// along O through a shared-memory transpose, or directly along I when the
// destination is also contiguous there.  Every thread keeps PERM_TO / 8 loads
// in flight so that enough bytes are outstanding per SM to cover HBM latency.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.h"
#include "ptx.cuh"

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
  } else if constexpr (MODE == PERM_F16X2) {
    const __half hi = __float2half_rn((float)v);
    reinterpret_cast<__half*>(dst0)[idx] = hi;
    reinterpret_cast<__half*>(dst1)[idx] = __float2half_rn((float)v - __half2float(hi));
  } else {
    __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
    reinterpret_cast<__nv_bfloat16*>(dst0)[idx] = hi;
    reinterpret_cast<__nv_bfloat16*>(dst1)[idx] = __float2bfloat16_rn((float)v - __bfloat162float(hi));
  }
}

constexpr int PT = 256;              // threads per CTA (register-staged kernel)

// Four consecutive outputs at a 4-element aligned index (vector stores).
template <typename Tin, int MODE>
__device__ __forceinline__ void put4(void* dst0, void* dst1, int64_t idx, Tin a, Tin b, Tin c, Tin d) {
  if constexpr (MODE == PERM_SAME && sizeof(Tin) == 8) {
    double2* p = reinterpret_cast<double2*>(reinterpret_cast<double*>(dst0) + idx);
    p[0] = make_double2((double)a, (double)b);
    p[1] = make_double2((double)c, (double)d);
  } else if constexpr (MODE == PERM_SAME) {
    *reinterpret_cast<float4*>(reinterpret_cast<float*>(dst0) + idx) = make_float4(a, b, c, d);
  } else if constexpr (MODE == PERM_TF32) {
    *reinterpret_cast<float4*>(reinterpret_cast<float*>(dst0) + idx) =
        make_float4(tf32_rna(a), tf32_rna(b), tf32_rna(c), tf32_rna(d));
  } else if constexpr (MODE == PERM_TF32X2) {
    const float ha = tf32_rna(a), hb = tf32_rna(b), hc = tf32_rna(c), hd = tf32_rna(d);
    *reinterpret_cast<float4*>(reinterpret_cast<float*>(dst0) + idx) = make_float4(ha, hb, hc, hd);
    *reinterpret_cast<float4*>(reinterpret_cast<float*>(dst1) + idx) =
        make_float4(tf32_rna(a - ha), tf32_rna(b - hb), tf32_rna(c - hc), tf32_rna(d - hd));
  } else if constexpr (MODE == PERM_F16X2) {
    const __half2 h01 = __floats2half2_rn(a, b), h23 = __floats2half2_rn(c, d);
    const float2 f01 = __half22float2(h01), f23 = __half22float2(h23);
    const __half2 l01 = __floats2half2_rn(a - f01.x, b - f01.y), l23 = __floats2half2_rn(c - f23.x, d - f23.y);
    uint2 hv, lv;
    hv.x = *reinterpret_cast<const uint32_t*>(&h01);
    hv.y = *reinterpret_cast<const uint32_t*>(&h23);
    lv.x = *reinterpret_cast<const uint32_t*>(&l01);
    lv.y = *reinterpret_cast<const uint32_t*>(&l23);
    *reinterpret_cast<uint2*>(reinterpret_cast<__half*>(dst0) + idx) = hv;
    *reinterpret_cast<uint2*>(reinterpret_cast<__half*>(dst1) + idx) = lv;
  } else {
    const __nv_bfloat162 h01 = __floats2bfloat162_rn(a, b), h23 = __floats2bfloat162_rn(c, d);
    uint2 hv;
    hv.x = *reinterpret_cast<const uint32_t*>(&h01);
    hv.y = *reinterpret_cast<const uint32_t*>(&h23);
    *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(dst0) + idx) = hv;
    if constexpr (MODE == PERM_BF16X2) {
      const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
      const __nv_bfloat162 l01 = __floats2bfloat162_rn(a - f01.x, b - f01.y);
      const __nv_bfloat162 l23 = __floats2bfloat162_rn(c - f23.x, d - f23.y);
      uint2 lv;
      lv.x = *reinterpret_cast<const uint32_t*>(&l01);
      lv.y = *reinterpret_cast<const uint32_t*>(&l23);
      *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(dst1) + idx) = lv;
    }
  }
}
constexpr int PR = PERM_TO / (PT / 32);  // rows per thread in a phase

template <typename Tin, int MODE>
__global__ void __launch_bounds__(PT) perm_kernel(const PermJob* __restrict__ jobs, int njobs, int64_t tiles,
                                                  const Tin* __restrict__ src0, const Tin* __restrict__ src1,
                                                  void* __restrict__ dst0, void* __restrict__ dst1) {
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
    const Tin* __restrict__ src = j->src_sel ? src1 : src0;
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


// ---------------------------------------------------------------------------------
// Shared-memory-staged sign-permute
struct StageMeta {
  int64_t baseD;
  int32_t nrows, ncols;
  int32_t ti, fast_i;
  int32_t sign, vec4;
  int32_t iwrite, qw, qp, wsuf;
};

constexpr int SPW = 6;                   // writer warps of the staged kernel
constexpr int SPP = 2;                   // producer warps (alternate tiles)
constexpr int SPT = 32 * (SPW + SPP);    // its threads

template <typename Tin>
struct StagedCfg {
  static constexpr int V = 16 / (int)sizeof(Tin);
  static constexpr int TE = PERM_TILE_BYTES / (int)sizeof(Tin);
  static constexpr int MAXTI = TE / 8;
  static constexpr int STAGE_ELEMS = TE + PERM_MAX_ROWS * V;
  static constexpr int BYTES = PERM_STAGES * STAGE_ELEMS * (int)sizeof(Tin) + PERM_STAGES * PERM_MAX_ROWS * (8 + 4) +
                               PERM_STAGES * MAXTI * (4 + 2 + 2) + PERM_STAGES * (int)sizeof(StageMeta) +
                               SPP * ((int)sizeof(PermJob) + (MAXR + 2) * 8) + 2 * PERM_STAGES * 8 + 128;
};

// Exact division of 0 <= x < 2^31 by an invariant d >= 1 with a multiply and
// a shift (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994): with l = ceil(log2 d), p = 31 + l and
// m = ceil(2^p / d) < 2^32, x / d = (x m) >> p, because m d - 2^p < d <= 2^l
// keeps the error term below 1 for every x < 2^31.
struct FastDiv {
  uint32_t m;
  int32_t p;
};

__device__ __forceinline__ FastDiv make_fastdiv(uint32_t d) {
  const int l = d > 1 ? 32 - __clz(d - 1) : 0;
  FastDiv f;
  f.p = 31 + l;
  f.m = (uint32_t)(((1ull << f.p) + d - 1) / d);
  return f;
}

__device__ __forceinline__ int32_t fdiv(int32_t x, FastDiv f) {
  return (int32_t)(((uint64_t)(uint32_t)x * f.m) >> f.p);
}

// The job of the tiles being staged, in shared memory: its record and the
// divisors of its leg dimensions and tile counts.
struct JobView {
  PermJob j;
  FastDiv leg[MAXR];
  FastDiv per_b, tiles_i;
};

static_assert(sizeof(PermJob) % 8 == 0, "jobs are copied as 8-byte words");

// Copy job `jn` into the view (the lanes of one warp).
__device__ __forceinline__ void load_job(const PermJob* __restrict__ jn, JobView* jv, int tid) {
  static_assert(MAXR + 2 <= 32, "one lane per divisor");
  const uint64_t* from = reinterpret_cast<const uint64_t*>(jn);
  uint64_t* to = reinterpret_cast<uint64_t*>(&jv->j);
  for (int w = tid; w < (int)(sizeof(PermJob) / 8); w += 32) to[w] = from[w];
  if (tid < MAXR) {
    const int nl = jn->nI + jn->nO + jn->nB;
    jv->leg[tid] = make_fastdiv(tid < nl ? (uint32_t)jn->dim[tid] : 1u);
  } else if (tid == MAXR) {
    jv->per_b = make_fastdiv((uint32_t)(jn->tiles_i * jn->tiles_o));
  } else if (tid == MAXR + 1) {
    jv->tiles_i = make_fastdiv((uint32_t)jn->tiles_i);
  }
}

// Where tile t of the job lies: its I and O ranges and the source and
// destination offsets of its batch index.  32-bit index arithmetic unless the
// job's tile count needs more.
struct TileGeo {
  int64_t bS, bD;
  int32_t i0, o0, ncols, nrows;
};

__device__ __forceinline__ TileGeo tile_geo(const JobView& v, int64_t t) {
  const PermJob& j = v.j;
  TileGeo g;
  const int64_t local = t - j.tile_begin;
  const int32_t tiles_i = j.tiles_i, per_b = tiles_i * j.tiles_o;
  int64_t b64;
  int32_t rem;
  if (local <= INT32_MAX) {
    const int32_t l32 = (int32_t)local, b32 = fdiv(l32, v.per_b);
    rem = l32 - b32 * per_b;
    b64 = b32;
  } else {
    b64 = local / per_b;
    rem = (int32_t)(local - b64 * per_b);
  }
  const int32_t to = fdiv(rem, v.tiles_i);
  g.i0 = (rem - to * tiles_i) * j.ti;
  g.o0 = to * j.tr;
  g.ncols = min(j.ti, j.PI - g.i0);
  g.nrows = min(j.tr, j.PO - g.o0);
  int64_t bS = j.src_off, bD = j.dst_off;
  const int nIO = j.nI + j.nO;
  if (b64 <= INT32_MAX) {
    int32_t x = (int32_t)b64;
    for (int q = nIO + j.nB - 1; q >= nIO; --q) {
      const int32_t qq = fdiv(x, v.leg[q]), idx = x - qq * j.dim[q];
      x = qq;
      bS += (int64_t)idx * j.sstr[q];
      bD += (int64_t)idx * j.dstr[q];
    }
  } else {
    int64_t x = b64;
    for (int q = nIO + j.nB - 1; q >= nIO; --q) {
      const int64_t d = j.dim[q], qq = x / d, idx = x - qq * d;
      x = qq;
      bS += idx * j.sstr[q];
      bD += idx * j.dstr[q];
    }
  }
  g.bS = bS;
  g.bD = bD;
  return g;
}

// The job of tile t, found by each warp for itself (tiles only move forward
// within a CTA, so the job index does too; next_begin caches where the next
// job starts, so most tiles touch no table).
__device__ __forceinline__ int find_job(const PermJob* __restrict__ jobs, int njobs, int64_t tiles, int64_t t, int nj,
                                        int64_t& next_begin, int lane) {
  if (nj >= 0 && t < next_begin) return nj;
  if (nj < 0) {
    // 32-way search: each round the lanes sample the window at 32 evenly
    // spaced jobs and keep the stretch after the last one starting at or
    // before t (a window of w jobs shrinks to ceil(w / 32) per round trip)
    int lo = 0, w = njobs;
    while (w > 1) {
      const int step = (w + 31) / 32;
      const int q = lo + lane * step;
      const unsigned ball = __ballot_sync(0xffffffffu, q < lo + w && jobs[q].tile_begin <= t);
      const int last = 31 - __clz(ball);  // lane 0 samples job lo, which starts at or before t
      lo += last * step;
      w = min(step, njobs - lo);
    }
    nj = lo;
  } else {
    // forward scan, 32 jobs per round (tile_begin increases with the job)
    for (;;) {
      const int q = nj + 1 + lane;
      const unsigned ball = __ballot_sync(0xffffffffu, q < njobs && jobs[q].tile_begin <= t);
      if (ball == 0) break;
      nj += 32 - __clz(ball);
      if (ball != 0xffffffffu) break;
    }
  }
  next_begin = nj + 1 < njobs ? jobs[nj + 1].tile_begin : tiles;
  return nj;
}

// The tables of tile t in its stage (the lanes of one producer warp take
// rows and columns in turn).
template <typename Tin>
__device__ __forceinline__ void stage_tables(const JobView& v, const TileGeo& g, int64_t* rowS, int32_t* rowD,
                                             int32_t* colD, int16_t* colS, int16_t* colP, StageMeta* meta, int tid) {
  const PermJob& j = v.j;
  const int nI = j.nI, nO = j.nO;
  for (int r = tid; r < g.nrows; r += 32) {
    int32_t x = g.o0 + r;
    int64_t rs = 0;
    int32_t rd = 0;
    for (int q = nI + nO - 1; q >= nI; --q) {
      const int32_t qq = fdiv(x, v.leg[q]), idx = x - qq * j.dim[q];
      x = qq;
      rs += (int64_t)idx * j.sstr[q];
      rd += idx * (int32_t)j.dstr[q];
    }
    rowS[r] = rs;
    rowD[r] = rd;
  }
  const int tc = tid;
  int32_t qp = 1;
  if (j.iwrite) {
    // the whole I group is in the tile (i0 = 0).  W (the destination run):
    // colS[q] = source column of the q-th element of the run (its legs'
    // destination strides are the run's own mixed radix).  P (the other I
    // legs, last fastest): colP[p] = source column, colD[p] = destination
    // offset of the p-th combination.
    const int32_t wmask = j.wmask, qw = j.qw;
    for (int q = tc; q < qw; q += 32) {
      int32_t cs = 0;
      for (int l = 0; l < nI; ++l)
        if (wmask >> l & 1) cs += ((q / (int32_t)j.dstr[l]) % j.dim[l]) * (int32_t)j.sstr[l];
      colS[q] = (int16_t)cs;
    }
    qp = g.ncols / qw;
    for (int p = tc; p < qp; p += 32) {
      int32_t x = p, cs = 0, dd = 0;
      for (int l = nI - 1; l >= 0; --l) {
        if (wmask >> l & 1) continue;
        const int32_t qq = fdiv(x, v.leg[l]), idx = x - qq * j.dim[l];
        x = qq;
        cs += idx * (int32_t)j.sstr[l];
        dd += idx * (int32_t)j.dstr[l];
      }
      colP[p] = (int16_t)cs;
      colD[p] = dd;
    }
  } else {
    for (int c = tc; c < g.ncols; c += 32) {
      int32_t x = g.i0 + c, dd = 0;
      for (int q = nI - 1; q >= 0; --q) {
        const int32_t qq = fdiv(x, v.leg[q]), idx = x - qq * j.dim[q];
        x = qq;
        dd += idx * (int32_t)j.dstr[q];
      }
      colD[c] = dd;
    }
  }
  if (tid == 0) {
    meta->baseD = g.bD;
    meta->nrows = g.nrows;
    meta->ncols = g.ncols;
    meta->ti = j.ti;
    meta->fast_i = j.store_fast_i;
    meta->sign = j.sign;
    meta->vec4 = j.vec4;
    meta->iwrite = j.iwrite;
    meta->qw = j.qw;
    meta->qp = qp;
    meta->wsuf = j.wsuf;
  }
}

// The tile's source rows into its stage: 16-byte chunks, consecutive lanes of
// the producer warp on consecutive chunks of a row (rows start 16-byte
// aligned, their lengths are multiples of 16 bytes).
template <typename Tin>
__device__ __forceinline__ void stage_copies(const Tin* __restrict__ src, const TileGeo& g, int ti, Tin* buf,
                                             const int64_t* rowS, int tid) {
  constexpr int V = StagedCfg<Tin>::V;
  const int cpr = g.ncols / V, stride = ti + V, nch = g.nrows * cpr;
  const Tin* sb = src + g.bS + g.i0;
  if ((cpr & (cpr - 1)) == 0) {
    const int sh = __ffs(cpr) - 1;
    for (int q = tid; q < nch; q += 32) {
      const int r = q >> sh, c = q & (cpr - 1);
      cp_async16(buf + r * stride + c * V, sb + rowS[r] + c * V);
    }
  } else {
    for (int q = tid; q < nch; q += 32) {
      const int r = q / cpr, c = q - r * cpr;
      cp_async16(buf + r * stride + c * V, sb + rowS[r] + c * V);
    }
  }
}

template <typename Tin, int MODE>
__global__ void __launch_bounds__(SPT, 3) perm_staged_kernel(const PermJob* __restrict__ jobs, int njobs, int64_t tiles,
                                                             const Tin* __restrict__ src, const Tin* __restrict__ src1,
                                                             void* __restrict__ dst0, void* __restrict__ dst1, int* err) {
  using Cfg = StagedCfg<Tin>;
  extern __shared__ uint8_t sm_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(sm_raw) + 127) & ~uintptr_t(127));
  Tin* buf = reinterpret_cast<Tin*>(sm);
  int64_t* rowS = reinterpret_cast<int64_t*>(buf + PERM_STAGES * Cfg::STAGE_ELEMS);
  int32_t* rowD = reinterpret_cast<int32_t*>(rowS + PERM_STAGES * PERM_MAX_ROWS);
  int32_t* colD = rowD + PERM_STAGES * PERM_MAX_ROWS;
  int16_t* colS = reinterpret_cast<int16_t*>(colD + PERM_STAGES * Cfg::MAXTI);
  int16_t* colP = colS + PERM_STAGES * Cfg::MAXTI;
  StageMeta* meta = reinterpret_cast<StageMeta*>(colP + PERM_STAGES * Cfg::MAXTI);
  JobView* jv = reinterpret_cast<JobView*>(meta + PERM_STAGES);
  uint64_t* full = reinterpret_cast<uint64_t*>(jv + SPP);
  uint64_t* empty = full + PERM_STAGES;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < PERM_STAGES; ++s) {
      mbar_init(&full[s], 64);    // the producing warp's lanes: tables written (32), copies landed (32)
      mbar_init(&empty[s], SPW);  // one per writer warp
    }
    fence_mbar_init();
  }
  __syncthreads();
  // Each CTA takes one contiguous range of tiles (the ranges differ in length
  // by at most one), so that consecutive tiles mostly belong to the same job.
  const int64_t t_first = (int64_t)blockIdx.x * tiles / gridDim.x;
  const int64_t n = ((int64_t)blockIdx.x + 1) * tiles / gridDim.x - t_first;
  if (warp >= SPW) {
    // ---- producer warps: tile k = p, p + SPP, ...: wait for its slot, build
    // its tables, copy its source rows (the lanes' cp.async copies arrive on
    // the slot's mbarrier when they land)
    const int pw = warp - SPW;
    JobView* v = jv + pw;
    int nj = -1, loaded = -1;
    int64_t next_begin = 0;
    bool first = true;
    for (int64_t k = pw; k < n; k += SPP) {
      const int s = (int)(k % PERM_STAGES);
      const uint32_t par = (uint32_t)((k / PERM_STAGES) & 1);
      bool ok = true;
      if (lane == 0) ok = mbar_wait(&empty[s], par ^ 1, err);
      __syncwarp();  // the writers' reads of the slot come before this warp's writes
      if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;
      const int64_t t = t_first + k;
      nj = find_job(jobs, njobs, tiles, t, nj, next_begin, lane);
      if (nj != loaded) {
        load_job(jobs + nj, v, lane);
        __syncwarp();
        loaded = nj;
      }
      const TileGeo g = tile_geo(*v, t);
      stage_tables<Tin>(*v, g, rowS + s * PERM_MAX_ROWS, rowD + s * PERM_MAX_ROWS, colD + s * Cfg::MAXTI,
                        colS + s * Cfg::MAXTI, colP + s * Cfg::MAXTI, meta + s, lane);
      const int ti = v->j.ti;
      const Tin* __restrict__ from = v->j.src_sel ? src1 : src;
      __syncwarp();  // every lane's row offsets are in rowS
      if (first) {
        // tensors are touched from here on (the job table and the tables
        // above are not written by kernels): wait for the grid before this
        // one (launched with programmatic serialisation), then let the next
        // one start
        pdl_wait();
        if (pw == 0 && lane == 0) pdl_launch_dependents();
        first = false;
      }
      mbar_arrive(&full[s]);  // this lane's table entries are written
      stage_copies<Tin>(from, g, ti, buf + s * Cfg::STAGE_ELEMS, rowS + s * PERM_MAX_ROWS, lane);
      cp_async_mbar_arrive_noinc(&full[s]);  // ... and its copies have landed
    }
    // no copy of this warp may still be landing when the CTA's shared memory
    // is released (after an early exit the writers no longer wait for them)
    cp_async_wait_all();
    return;
  }
  // ---- writer warps: tile k once its slot is full, then release the slot
  bool first = true;
  for (int64_t k = 0; k < n; ++k) {
    const int s = (int)(k % PERM_STAGES);
    const uint32_t par = (uint32_t)((k / PERM_STAGES) & 1);
    if (!mbar_wait(&full[s], par, err)) break;
    if (first) {  // before the first store (the previous grid has completed)
      pdl_wait();
      first = false;
    }
    const StageMeta m = meta[s];
    const Tin* tb = buf + s * Cfg::STAGE_ELEMS;
    const int32_t* rd = rowD + s * PERM_MAX_ROWS;
    const int32_t* cd = colD + s * Cfg::MAXTI;
    const int stride = m.ti + Cfg::V;
    const Tin sgn = (Tin)m.sign;
    if (m.iwrite) {
      // destination order along I: every (row, P) pair owns a contiguous run
      // of qw destination elements, gathered from the stage by colS (or read
      // straight when the run is the innermost I legs in order)
      const int16_t* csw = colS + s * Cfg::MAXTI;
      const int16_t* csp = colP + s * Cfg::MAXTI;
      const int npairs = m.nrows * m.qp;
      const int qps = (m.qp & (m.qp - 1)) == 0 ? __ffs(m.qp) - 1 : -1;
      const int vq = m.vec4 ? 4 : 1, units = m.qw / vq;
      const bool grouped = units < 32 && (units & (units - 1)) == 0;
      const int lg = grouped ? __ffs(units) - 1 : 5, per = grouped ? 32 >> lg : 1;
      const int sub = grouped ? lane >> lg : 0;
      const int q0 = grouped ? (lane & (units - 1)) * vq : lane * vq;
      const int qstep = grouped ? m.qw : 32 * vq;
      for (int rp0 = warp * per; rp0 < npairs; rp0 += SPW * per) {
        const int rp = rp0 + sub;
        if (rp >= npairs) continue;
        int r, p;
        if (qps >= 0) {
          r = rp >> qps;
          p = rp & (m.qp - 1);
        } else {
          r = rp / m.qp;
          p = rp - r * m.qp;
        }
        const Tin* x = tb + r * stride + csp[p];
        const int64_t base = m.baseD + rd[r] + cd[p];
        for (int q = q0; q < m.qw; q += qstep) {
          if (vq == 4) {
            Tin a, b, c, d;
            if (m.wsuf) {
              a = x[q], b = x[q + 1], c = x[q + 2], d = x[q + 3];
            } else {
              a = x[csw[q]], b = x[csw[q + 1]], c = x[csw[q + 2]], d = x[csw[q + 3]];
            }
            put4<Tin, MODE>(dst0, dst1, base + q, sgn * a, sgn * b, sgn * c, sgn * d);
          } else {
            put<Tin, MODE>(dst0, dst1, base + q, sgn * x[m.wsuf ? q : csw[q]]);
          }
        }
      }
    } else if (m.vec4 && m.fast_i) {
      // quads of consecutive I elements, contiguous in the destination
      for (int r = warp; r < m.nrows; r += SPW) {
        const int64_t base = m.baseD + rd[r];
        for (int c4 = 4 * lane; c4 < m.ncols; c4 += 128) {
          const Tin* x = tb + r * stride + c4;
          put4<Tin, MODE>(dst0, dst1, base + cd[c4], sgn * x[0], sgn * x[1], sgn * x[2], sgn * x[3]);
        }
      }
    } else if (m.fast_i) {
      for (int r = warp; r < m.nrows; r += SPW) {
        const int64_t base = m.baseD + rd[r];
        for (int c = lane; c < m.ncols; c += 32) put<Tin, MODE>(dst0, dst1, base + cd[c], sgn * tb[r * stride + c]);
      }
    } else {
      for (int c0 = warp * Cfg::V; c0 < m.ncols; c0 += SPW * Cfg::V) {
        for (int r = lane; r < m.nrows; r += 32) {
          Tin v[Cfg::V];
          if constexpr (sizeof(Tin) == 4) {
            const float4 w = *reinterpret_cast<const float4*>(tb + r * stride + c0);
            v[0] = w.x, v[1] = w.y, v[2] = w.z, v[3] = w.w;
          } else {
            const double2 w = *reinterpret_cast<const double2*>(tb + r * stride + c0);
            v[0] = w.x, v[1] = w.y;
          }
          const int64_t base = m.baseD + rd[r];
#pragma unroll
          for (int q = 0; q < Cfg::V; ++q)
            if (c0 + q < m.ncols) put<Tin, MODE>(dst0, dst1, base + cd[c0 + q], sgn * v[q]);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

template <typename Tin, int MODE>
static cudaError_t go_staged(ftn_ctx ctx, const PermJob* d_jobs, int njobs, int64_t tiles, const void* src,
                             const void* src1, void* dst0, void* dst1) {
  using Cfg = StagedCfg<Tin>;
  static const cudaError_t attr =
      cudaFuncSetAttribute(perm_staged_kernel<Tin, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::BYTES);
  if (attr != cudaSuccess) return attr;
  int64_t grid = tiles;
  int64_t cap = (int64_t)ctx->num_sms * 3;
  if (grid > cap) grid = cap;
  return launch_pdl(perm_staged_kernel<Tin, MODE>, (unsigned)grid, SPT, Cfg::BYTES, ctx->stream, d_jobs, njobs, tiles,
                    (const Tin*)src, (const Tin*)src1, dst0, dst1, ctx->dev_err);
}

template <typename Tin, int MODE>
static cudaError_t go(ftn_ctx ctx, const PermJob* d_jobs, int njobs, int64_t tiles, const void* src,
                      const void* src1, void* dst0, void* dst1) {
  int64_t grid = tiles;
  int64_t cap = (int64_t)ctx->num_sms * 16;
  if (grid > cap) grid = cap;
  perm_kernel<Tin, MODE><<<(unsigned)grid, PT, 0, ctx->stream>>>(d_jobs, njobs, tiles, (const Tin*)src,
                                                                  (const Tin*)src1, dst0, dst1);
  return cudaGetLastError();
}

template <typename Tin, int MODE>
static cudaError_t pick(ftn_ctx ctx, int staged, const PermJob* d_jobs, int njobs, int64_t tiles, const void* src,
                        const void* src1, void* dst0, void* dst1) {
  return staged ? go_staged<Tin, MODE>(ctx, d_jobs, njobs, tiles, src, src1, dst0, dst1)
                : go<Tin, MODE>(ctx, d_jobs, njobs, tiles, src, src1, dst0, dst1);
}

ftn_status launch_permute2(ftn_ctx ctx, const PermJob* d_jobs, int njobs, int64_t tiles, int staged, const void* src,
                           const void* src1, void* dst0, void* dst1, ftn_dtype in_type, int mode) {
  if (njobs == 0 || tiles == 0) return FTN_OK;
  cudaError_t e;
  if (in_type == FTN_F64) {
    if (mode != PERM_SAME) return set_error(FTN_EUNSUPPORTED, "FP64 permute supports only the same-type output");
    e = pick<double, PERM_SAME>(ctx, staged, d_jobs, njobs, tiles, src, src1, dst0, dst1);
  } else {
    switch (mode) {
      case PERM_SAME: e = pick<float, PERM_SAME>(ctx, staged, d_jobs, njobs, tiles, src, src1, dst0, dst1); break;
      case PERM_TF32: e = pick<float, PERM_TF32>(ctx, staged, d_jobs, njobs, tiles, src, src1, dst0, dst1); break;
      case PERM_TF32X2: e = pick<float, PERM_TF32X2>(ctx, staged, d_jobs, njobs, tiles, src, src1, dst0, dst1); break;
      case PERM_BF16: e = pick<float, PERM_BF16>(ctx, staged, d_jobs, njobs, tiles, src, src1, dst0, dst1); break;
      case PERM_BF16X2: e = pick<float, PERM_BF16X2>(ctx, staged, d_jobs, njobs, tiles, src, src1, dst0, dst1); break;
      case PERM_F16X2: e = pick<float, PERM_F16X2>(ctx, staged, d_jobs, njobs, tiles, src, src1, dst0, dst1); break;
      default: return set_error(FTN_EINVAL, "bad permute mode");
    }
  }
  ctx->launches += 1;
  if (e != cudaSuccess) return cuda_error(e, "perm_kernel launch");
  return FTN_OK;
}

ftn_status launch_permute(ftn_ctx ctx, const PermJob* d_jobs, int njobs, int64_t tiles, int staged, const void* src,
                          void* dst0, void* dst1, ftn_dtype in_type, int mode) {
  return launch_permute2(ctx, d_jobs, njobs, tiles, staged, src, src, dst0, dst1, in_type, mode);
}

}  // namespace ftn
