// Grouped sector GEMM on the tcgen05 tensor cores (sm_103a).
//
// One persistent launch covers every (row block, column block) problem of a
// fermionic contraction: C_blk[m, n] = sum_k A_pi[row0 + m, k] B_pi[col0 + n, k]
// where A_pi / B_pi are the fused sector matrices of bond parity pi (K-major,
// produced by the sign-permute kernel).  Warp roles per CTA:
//   warp 0    TMA producer: 128 x 32 (TF32) or 128 x 64 (BF16 / FP16) A tiles and
//             BN x same B tiles into a STAGES-deep shared-memory ring;
//   warp 1    MMA issuer: tcgen05.mma (M = 128, N = BN) into one of two TMEM
//             accumulators, tcgen05.commit releases ring slots;
//   warps 2-9 epilogue, two sets of four (one per TMEM accumulator buffer):
//             tcgen05.ld of the accumulator (one row per thread), FP32
//             stores into the output block.
// Split modes (TF32X3 / BF16X3 / F16X3) load hi and lo planes; hi*hi goes into one
// TMEM accumulator and hi*lo + lo*hi into a second one, summed in FP32 by the
// epilogue.  The tensor core's accumulation rounds each partial sum, so
// keeping the large products apart from the two small cross terms cuts the
// number of roundings applied to the large accumulator by three.
#include <algorithm>
#include <cstddef>
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.h"
#include "ptx.cuh"

namespace ftn {

constexpr int TC_BM = 128;
constexpr int TC_EPI_WARPS = 8;  // two sets of four, one per TMEM accumulator buffer
constexpr int TC_THREADS = 64 + 32 * TC_EPI_WARPS;

struct TcParams {
  CUtensorMap a_hi[2];
  CUtensorMap b_hi[2];
  CUtensorMap a_lo[2];
  CUtensorMap b_lo[2];
  // Batched launches (problems of many contractions): when set, problem p
  // reads its operands through gmaps[4 * p.pi + {0: A hi, 1: B hi, 2: A lo,
  // 3: B lo}] (global memory, 64-byte aligned) instead of the maps above.
  const CUtensorMap* gmaps;
  const TileEnt* tt;  // decoded tiles (or null: decode with tc_decode)
  const GemmProb* probs;
  float* C;
  int* err;
  int64_t tiles;
  int nprobs;
  int contig;  // 1: each CTA takes a contiguous range of tiles (else a strided set)
};

// FMT: operand format, the instruction descriptor's code (0 = FP16, 1 = BF16
// with kind::f16; 2 = TF32 with kind::tf32); A and B always share it.
template <int FMT, bool SPLIT, int BN>
struct TcCfg {
  static constexpr bool HALF = FMT != 2;
  static constexpr int A_BYTES = TC_BM * 128;
  static constexpr int B_BYTES = BN * 128;
  static constexpr int OPS = SPLIT ? 2 : 1;
  static constexpr int STAGE_BYTES = (A_BYTES + B_BYTES) * OPS;
  // epilogue staging: per epilogue warp a 32 x (CW + 1) FP32 tile
  static constexpr int CW = BN < 32 ? BN : 32;
  static constexpr int EPI_BYTES = TC_EPI_WARPS * 32 * (CW + 1) * 4;
  static constexpr int BUDGET = 227 * 1024 - 1024 - 256 - EPI_BYTES;
  static constexpr int STAGES_RAW = BUDGET / STAGE_BYTES;
  static constexpr int STAGES = STAGES_RAW > 8 ? 8 : STAGES_RAW;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256 + EPI_BYTES;
  // two accumulator buffers; split modes keep the hi*hi products and the
  // small cross terms in separate accumulators (ACC_W columns per buffer)
  static constexpr int ACC_W = SPLIT ? 2 * BN : BN;
  static constexpr int TMEM_COLS = (2 * ACC_W < 32) ? 32 : 2 * ACC_W;
  static constexpr int KB = HALF ? 64 : 32;  // K elements per stage (128 B)
  static constexpr uint32_t IDESC = idesc_f32acc(TC_BM, BN, (uint32_t)FMT);
  static_assert(STAGES >= 2, "shared memory ring too shallow");
};

__device__ __forceinline__ int tc_find_prob(const GemmProb* probs, int nprobs, int64_t t) {
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

// Tile t -> (problem, m0, n0) under the grouped order (see GemmProb).  A
// CTA's tiles increase, so `cur` (the group found for the previous tile, -1
// at the start) only moves forward: one look at the next group's first
// tile instead of a binary search of the table per tile.
template <int BN>
__device__ __forceinline__ const GemmProb* tc_decode(const TcParams& P, int64_t t, int& m0, int& n0, int& cur) {
  if (cur < 0) {
    cur = tc_find_prob(P.probs, P.nprobs, t);
    cur = P.probs[cur].grp_first;
  } else {
    for (;;) {
      const int nxt = P.probs[cur].grp_first + P.probs[cur].grp_count;
      if (nxt >= P.nprobs || P.probs[nxt].tile_begin > t) break;
      cur = nxt;
    }
  }
  const GemmProb* g = P.probs + cur;
  const int64_t local = t - g->tile_begin;
  const int tm = (int)(local / g->row_tiles);
  int rem = (int)(local - (int64_t)tm * g->row_tiles);
  const GemmProb* p = P.probs + g->grp_first;
  if (g->gmerge) {  // column n0 counts across the group's members
    m0 = tm * TC_BM;
    n0 = rem * BN;
    return p;
  }
  for (int q = 0; q < g->grp_count; ++q, ++p)
    if (rem < p->tn_off + p->tiles_n) break;
  m0 = tm * TC_BM;
  n0 = (rem - p->tn_off) * BN;
  return p;
}

// Tile t as a TileEnt: from the launch's tile table when there is one (one
// 32-byte load), else decoded here (`cur` as for tc_decode).
template <int BN>
__device__ __forceinline__ void tile_at(const TcParams& P, int64_t t, int& cur, TileEnt& e) {
  if (P.tt) {
    const int4* q = reinterpret_cast<const int4*>(P.tt + t);
    const int4 a = q[0], b = q[1];
    e.prob = a.x, e.m0 = a.y, e.n0 = a.z, e.pi = a.w;
    e.a_y = b.x, e.b_y = b.y, e.K = b.z, e.k0 = b.w;
    return;
  }
  int m0, n0;
  const GemmProb* p = tc_decode<BN>(P, t, m0, n0, cur);
  e.prob = (int32_t)(p - P.probs);
  e.m0 = m0;
  e.n0 = n0;
  e.pi = p->pi;
  e.a_y = p->a_row0 + m0;
  e.b_y = p->b_row0 + n0;
  e.K = p->K;
  e.k0 = p->k0;
}

template <int BN>
__global__ void tile_table_kernel(TcParams P, TileEnt* __restrict__ out) {
  P.tt = nullptr;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < P.tiles; t += (int64_t)gridDim.x * blockDim.x) {
    int cur = -1;
    TileEnt e;
    tile_at<BN>(P, t, cur, e);
    out[t] = e;
  }
}

template <int FMT, bool SPLIT, int BN>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(const __grid_constant__ TcParams P) {
  using Cfg = TcCfg<FMT, SPLIT, BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Cfg::STAGES * Cfg::STAGE_BYTES);
  uint64_t* empty = full + Cfg::STAGES;
  uint64_t* tfull = empty + Cfg::STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  float* epi = reinterpret_cast<float*>(smem + Cfg::STAGES * Cfg::STAGE_BYTES + 256);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 4);
    }
    mbar_init(drain, 1);
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tslot, Cfg::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  // This CTA's tiles: one contiguous range when the launch has many tiles per
  // CTA (the ranges differ in length by at most one; consecutive tiles then
  // mostly share their problem, so the epilogue keeps its records and column
  // offsets in registers), else every gridDim.x-th tile (concurrent CTAs then
  // work on neighbouring tiles, whose operand rows and columns they share in
  // L2).
  const int64_t t_begin = P.contig ? (int64_t)blockIdx.x * P.tiles / gridDim.x : (int64_t)blockIdx.x;
  const int64_t t_step = P.contig ? 1 : (int64_t)gridDim.x;
  const int64_t n_my = P.contig ? ((int64_t)blockIdx.x + 1) * P.tiles / gridDim.x - t_begin
                                : (P.tiles - blockIdx.x + gridDim.x - 1) / gridDim.x;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued = 0, lastpar = 0;
      bool ok = true;
      int cur = -1, fenced = -1;
      TileEnt nx;
      if (n_my > 0) tile_at<BN>(P, t_begin, cur, nx);
      // the operands are read from here on (the tile and problem tables are
      // not written by kernels): wait for the grid before this one, then let
      // the next one start
      pdl_wait();
      pdl_launch_dependents();
      for (int64_t k = 0; k < n_my && ok; ++k) {
        const int64_t t = t_begin + k * t_step;
        const TileEnt e = nx;  // this tile; the next one's entry is fetched while this one is issued
        if (k + 1 < n_my) tile_at<BN>(P, t + t_step, cur, nx);
        const int nk = (e.K + Cfg::KB - 1) / Cfg::KB;
        const int pi = e.pi;
        const CUtensorMap *ma = &P.a_hi[pi & 1], *mb = &P.b_hi[pi & 1], *mal = &P.a_lo[pi & 1],
                          *mbl = &P.b_lo[pi & 1];
        if (P.gmaps) {
          ma = P.gmaps + 4 * pi;
          mb = ma + 1;
          mal = ma + 2;
          mbl = ma + 3;
          if (nk > 0 && fenced != pi) {
            tensormap_acquire(ma);
            tensormap_acquire(mb);
            if constexpr (SPLIT) {
              tensormap_acquire(mal);
              tensormap_acquire(mbl);
            }
            fenced = pi;
          }
        }
        for (int kb = 0; kb < nk; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1, P.err)) {
            ok = false;
            break;
          }
          uint8_t* sa = smem + stage * Cfg::STAGE_BYTES;
          mbar_expect_tx(&full[stage], Cfg::STAGE_BYTES);
          const int kx = e.k0 + kb * Cfg::KB;  // K element; k0 is a multiple of KB
          tma_load_2d(sa, ma, kx, e.a_y, &full[stage]);
          tma_load_2d(sa + Cfg::A_BYTES, mb, kx, e.b_y, &full[stage]);
          if constexpr (SPLIT) {
            tma_load_2d(sa + Cfg::A_BYTES + Cfg::B_BYTES, mal, kx, e.a_y, &full[stage]);
            tma_load_2d(sa + 2 * Cfg::A_BYTES + Cfg::B_BYTES, mbl, kx, e.b_y, &full[stage]);
          }
          issued |= 1u << stage;
          lastpar = (lastpar & ~(1u << stage)) | (phase << stage);
          if (++stage == Cfg::STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      // wait for this CTA's own copies still in flight
      for (int s = 0; s < Cfg::STAGES; ++s)
        if (issued & (1u << s)) mbar_wait(&full[s], (lastpar >> s) & 1, P.err, false);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool ok = true;
      int cur = -1;
      TileEnt nx;
      if (n_my > 0) tile_at<BN>(P, t_begin, cur, nx);
      for (int64_t k = 0; k < n_my && ok; ++k) {
        const int64_t t = t_begin + k * t_step;
        const TileEnt e = nx;
        if (k + 1 < n_my) tile_at<BN>(P, t + t_step, cur, nx);
        const int nk = (e.K + Cfg::KB - 1) / Cfg::KB;
        if (nk == 0) continue;
        if (!mbar_wait(&tempty[acc], acc_phase ^ 1, P.err)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * Cfg::ACC_W);
        const uint32_t d_small = d + (uint32_t)BN;
        for (int kb = 0; kb < nk; ++kb) {
          if (!mbar_wait(&full[stage], phase, P.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + stage * Cfg::STAGE_BYTES);
          const uint32_t sb = sa + Cfg::A_BYTES;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint64_t ad = sdesc_sw128(sa + 32 * j);
            const uint64_t bd = sdesc_sw128(sb + 32 * j);
            const uint32_t accum = (kb | j) != 0;
            if constexpr (Cfg::HALF)
              mma_f16(d, ad, bd, Cfg::IDESC, accum);
            else
              mma_tf32(d, ad, bd, Cfg::IDESC, accum);
            if constexpr (SPLIT) {
              const uint32_t sal = sa + Cfg::A_BYTES + Cfg::B_BYTES;
              const uint32_t sbl = sal + Cfg::A_BYTES;
              const uint64_t adl = sdesc_sw128(sal + 32 * j);
              const uint64_t bdl = sdesc_sw128(sbl + 32 * j);
              if constexpr (Cfg::HALF) {
                mma_f16(d_small, ad, bdl, Cfg::IDESC, accum);
                mma_f16(d_small, adl, bd, Cfg::IDESC, 1);
              } else {
                mma_tf32(d_small, ad, bdl, Cfg::IDESC, accum);
                mma_tf32(d_small, adl, bd, Cfg::IDESC, 1);
              }
            }
          }
          mma_commit(&empty[stage]);
          if (++stage == Cfg::STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        mma_commit(&tfull[acc]);
        acc ^= 1;
        if (acc == 0) acc_phase ^= 1;
      }
      // every issued MMA has completed before TMEM is released
      mma_commit(drain);
      mbar_wait(drain, 0, P.err, false);
    }
  } else {
    // ---------------- epilogue (warps 2..9) ----------------
    // Two sets of four warps; set s drains the tiles that used TMEM buffer s,
    // so two tiles are written out concurrently.  Within a set, warp w reads
    // TMEM lanes 32*(w%4)..+31 (one output row per lane).  TMEM -> registers
    // -> shared memory -> global, one 32-column chunk at a time, so that every
    // warp store writes 32 consecutive destination elements.  Output
    // addresses follow the problem's row/column leg tables (a permuted output
    // layout costs nothing extra here).
    const int q = warp & 3;
    const int set = (warp - 2) >> 2;
    float* stg = epi + (warp - 2) * 32 * (Cfg::CW + 1);
    uint32_t j = 0;  // tiles with K > 0 seen so far (all sets count them)
    const bool c16 = ((uintptr_t)P.C & 15) == 0;  // 16-byte vector stores need an aligned base
    int cur = -1;
    // tile entries two tiles ahead (a set writes every other tile out)
    TileEnt nx, nx2;
    if (n_my > 0) tile_at<BN>(P, t_begin, cur, nx);
    if (n_my > 1) tile_at<BN>(P, t_begin + t_step, cur, nx2);
    constexpr int NCH = BN / Cfg::CW;
    // The problem records of the last tile written out, kept in registers
    // while the tiles stay on the same problem and first column (in a
    // grouped launch most consecutive tiles do): lane l < MAXR holds row leg
    // l, MAXR <= l < 2 MAXR column leg l - MAXR, lanes 0..9 also the scalars
    // below (32-bit words of the record); mi: each chunk's member.
    bool waited = false;
    int key_prob = -1, key_n0 = -1;
    int gm = 0, pM = 0;
    int32_t ldim[NCH];
    int64_t lstr[NCH];
    // column side of each chunk (independent of the tile's rows), kept with
    // the records: column offset, valid columns, store mode, sign, the
    // member's output offset, rows and row legs; rows_same: every chunk's
    // member has the first one's row legs (one row expansion per tile)
    int64_t cp_c[NCH], coff_c[NCH];
    int cn_c[NCH], fl_c[NCH], mM_c[NCH], nrl_c[NCH];
    float sg_c[NCH];
    bool rows_same = true;
    for (int64_t k = 0; k < n_my; ++k) {
      const int64_t t = t_begin + k * t_step;
      const TileEnt e = nx;
      nx = nx2;
      if (k + 2 < n_my) tile_at<BN>(P, t + 2 * t_step, cur, nx2);
      const int m0 = e.m0, n0 = e.n0;
      const GemmProb* __restrict__ pp = P.probs + e.prob;
      const int nk = (e.K + Cfg::KB - 1) / Cfg::KB;
      const int acc = (int)(j & 1);
      if (nk > 0) ++j;
      if (nk > 0 ? acc != set : set != 0) continue;
      const int row = m0 + 32 * q + lane;
      // Per chunk of CW columns: its problem (a member of a merged group),
      // valid columns, this lane's row and column offsets, sign and store
      // mode.  When the tile's problem or first column differs from the last
      // one's, the records are read again, spread over the lanes and issued
      // together in two round trips (the group's member ends; then every
      // chunk's leg tables and scalars) before waiting for the accumulator:
      // walking the table with dependent reads for every tile cost more than
      // the tile's stores.
      int64_t rp_c[NCH];
      if (e.prob != key_prob || n0 != key_n0) {
        key_prob = e.prob;
        key_n0 = n0;
        gm = pp->gmerge;
        pM = pp->M;
        const int gc = pp->grp_count;
        const bool in_tab = e.prob + lane < P.nprobs;
        const int mg = in_tab ? pp[lane].gcol : 0, mn = in_tab ? pp[lane].N : 0;
        int mi[NCH];
        int32_t wsc[NCH];
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
          const int lcol = n0 + ch * Cfg::CW;
          int m = 0;
          if (gm) {
            if (gc <= 32) {
              // members are in column order: those ending at or before lcol
              m = __popc(__ballot_sync(0xffffffffu, lane < gc - 1 && lcol >= mg + mn));
            } else {
              const GemmProb* mp = pp;
              for (int qq = 1; qq < gc && lcol >= mp->gcol + mp->N; ++qq) ++mp;
              m = (int)(mp - pp);
            }
          }
          mi[ch] = m;
        }
        static_assert(2 * MAXR <= 32, "one warp holds the row and column legs");
        constexpr int W_COFF = (int)(offsetof(GemmProb, c_off) / 4), W_M = (int)(offsetof(GemmProb, M) / 4),
                      W_N = (int)(offsetof(GemmProb, N) / 4), W_SIGN = (int)(offsetof(GemmProb, c_sign) / 4),
                      W_NRL = (int)(offsetof(GemmProb, nrl) / 4), W_NCL = (int)(offsetof(GemmProb, ncl) / 4),
                      W_EROWS = (int)(offsetof(GemmProb, epi_rows) / 4), W_VEC4 = (int)(offsetof(GemmProb, vec4) / 4),
                      W_GCOL = (int)(offsetof(GemmProb, gcol) / 4);
        const int woff = lane == 0   ? W_COFF
                         : lane == 1 ? W_COFF + 1
                         : lane == 2 ? W_M
                         : lane == 3 ? W_N
                         : lane == 4 ? W_SIGN
                         : lane == 5 ? W_NRL
                         : lane == 6 ? W_NCL
                         : lane == 7 ? W_EROWS
                         : lane == 8 ? W_VEC4
                                     : W_GCOL;
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
          const GemmProb* __restrict__ mp = pp + mi[ch];
          ldim[ch] = 1;
          lstr[ch] = 0;
          wsc[ch] = 0;
          if (lane < MAXR) {
            ldim[ch] = mp->rdim[lane];
            lstr[ch] = mp->rstr[lane];
          } else if (lane < 2 * MAXR) {
            ldim[ch] = mp->cdim[lane - MAXR];
            lstr[ch] = mp->cstr[lane - MAXR];
          }
          if (lane < 10) wsc[ch] = reinterpret_cast<const int32_t*>(mp)[woff];
        }
        const uint32_t fm = 0xffffffffu;
        rows_same = true;
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
          coff_c[ch] = (int64_t)(uint32_t)__shfl_sync(fm, wsc[ch], 0) | ((int64_t)__shfl_sync(fm, wsc[ch], 1) << 32);
          mM_c[ch] = __shfl_sync(fm, wsc[ch], 2);
          const int mN = __shfl_sync(fm, wsc[ch], 3);
          const int csign = __shfl_sync(fm, wsc[ch], 4);
          nrl_c[ch] = __shfl_sync(fm, wsc[ch], 5);
          const int ncl = __shfl_sync(fm, wsc[ch], 6), erows = __shfl_sync(fm, wsc[ch], 7);
          const int vec4 = __shfl_sync(fm, wsc[ch], 8), gcol = __shfl_sync(fm, wsc[ch], 9);
          const int lcol = n0 + ch * Cfg::CW - (gm ? gcol : 0);
          const int cn = mN - lcol < Cfg::CW ? mN - lcol : Cfg::CW;
          cn_c[ch] = cn;
          cp_c[ch] = 0;
          sg_c[ch] = 1.0f;
          fl_c[ch] = 0;
          if (cn > 0) {
            int xc = lcol + lane;
            int64_t co = 0;
            for (int l = ncl - 1; l >= 0; --l) {
              const int d = __shfl_sync(fm, ldim[ch], MAXR + l);
              const int64_t st = __shfl_sync(fm, lstr[ch], MAXR + l);
              const int qq = xc / d;
              co += (int64_t)(xc - qq * d) * st;
              xc = qq;
            }
            cp_c[ch] = lane < Cfg::CW && lane < cn ? co : 0;
            sg_c[ch] = (float)csign;
            fl_c[ch] = (vec4 && c16 ? 1 : 0) | (erows ? 2 : 0);
          }
          if (ch > 0)
            rows_same = rows_same && nrl_c[ch] == nrl_c[0] &&
                        __all_sync(fm, lane >= MAXR || (ldim[ch] == ldim[0] && lstr[ch] == lstr[0]));
        }
      }
      const int nrows = pM - (m0 + 32 * q) < 32 ? pM - (m0 + 32 * q) : 32;
      {
        // row side: this lane's row within the member's output block
        const uint32_t fm = 0xffffffffu;
        int64_t r0 = 0;
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
          rp_c[ch] = 0;
          if (cn_c[ch] <= 0) continue;
          if (ch == 0 || !rows_same) {
            int x = row;
            int64_t ro = 0;
            for (int l = nrl_c[ch] - 1; l >= 0; --l) {
              const int d = __shfl_sync(fm, ldim[ch], l);
              const int64_t st = __shfl_sync(fm, lstr[ch], l);
              const int qq = x / d;
              ro += (int64_t)(x - qq * d) * st;
              x = qq;
            }
            r0 = ro;
          }
          rp_c[ch] = row < mM_c[ch] ? coff_c[ch] + r0 : 0;
        }
      }
      if (!waited) {  // the first store of C: the grid before this one has completed
        pdl_wait();
        waited = true;
      }
      if (nk > 0) {
        if (!mbar_wait(&tfull[acc], ((j - 1) >> 1) & 1, P.err)) break;
        tc_fence_after();
      }
      const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * Cfg::ACC_W);
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
        const int c = ch * Cfg::CW;
        const int cn = cn_c[ch];
        if (cn <= 0) break;
        const int64_t rpart = rp_c[ch];
        const float sg = sg_c[ch];
        float v[Cfg::CW];
        if (nk > 0) {
#pragma unroll
          for (int h = 0; h < Cfg::CW; h += 16) {
            uint32_t r[16];
            tmem_ld16(taddr + (uint32_t)(c + h), r);
            if constexpr (SPLIT) {
              uint32_t r2[16];
              tmem_ld16(taddr + (uint32_t)(BN + c + h), r2);
              tmem_wait_ld();
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) v[h + jj] = __uint_as_float(r[jj]) + __uint_as_float(r2[jj]);
            } else {
              tmem_wait_ld();
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) v[h + jj] = __uint_as_float(r[jj]);
            }
          }
        } else {
#pragma unroll
          for (int jj = 0; jj < Cfg::CW; ++jj) v[jj] = 0.0f;
        }
        const int64_t cpart = cp_c[ch];
#pragma unroll
        for (int jj = 0; jj < Cfg::CW; ++jj) stg[lane * (Cfg::CW + 1) + jj] = v[jj];
        __syncwarp();
        const bool okc = lane < Cfg::CW && lane < cn;
        if (fl_c[ch] & 1) {
          // 16-byte stores: quads of consecutive elements along the contiguous direction
          const int sub = lane & 7, grp = lane >> 3;
          if (fl_c[ch] & 2) {
            // lane -> rows 4*sub..+3 of column cc = 4*it + grp
            const int64_t rq = __shfl_sync(0xffffffffu, rpart, 4 * sub);
#pragma unroll
            for (int it = 0; it < Cfg::CW / 4; ++it) {
              const int cc = 4 * it + grp;
              const int64_t cp = __shfl_sync(0xffffffffu, cpart, cc);
              if (4 * sub < nrows && cc < cn) {
                float4 w;
                w.x = sg * stg[(4 * sub + 0) * (Cfg::CW + 1) + cc];
                w.y = sg * stg[(4 * sub + 1) * (Cfg::CW + 1) + cc];
                w.z = sg * stg[(4 * sub + 2) * (Cfg::CW + 1) + cc];
                w.w = sg * stg[(4 * sub + 3) * (Cfg::CW + 1) + cc];
                *reinterpret_cast<float4*>(P.C + rq + cp) = w;
              }
            }
          } else {
            // lane -> columns 4*sub..+3 (sub < CW/4) of row rr = 4*it + grp
            const int64_t cq = __shfl_sync(0xffffffffu, cpart, (4 * sub) & 31);
#pragma unroll
            for (int it = 0; it < 8; ++it) {
              const int rr = 4 * it + grp;
              const int64_t rp = __shfl_sync(0xffffffffu, rpart, rr);
              if (4 * sub < Cfg::CW && rr < nrows && 4 * sub < cn) {
                float4 w;
                w.x = sg * stg[rr * (Cfg::CW + 1) + 4 * sub + 0];
                w.y = sg * stg[rr * (Cfg::CW + 1) + 4 * sub + 1];
                w.z = sg * stg[rr * (Cfg::CW + 1) + 4 * sub + 2];
                w.w = sg * stg[rr * (Cfg::CW + 1) + 4 * sub + 3];
                *reinterpret_cast<float4*>(P.C + rp + cq) = w;
              }
            }
          }
        } else if (fl_c[ch] & 2) {
          // destination contiguous along rows: lane -> row, loop over columns
#pragma unroll 4
          for (int cc = 0; cc < Cfg::CW; ++cc) {
            const int64_t cp = __shfl_sync(0xffffffffu, cpart, cc);
            if (lane < nrows && cc < cn) P.C[rpart + cp] = sg * stg[lane * (Cfg::CW + 1) + cc];
          }
        } else {
#pragma unroll 4
          for (int rr = 0; rr < 32; ++rr) {
            const int64_t rp = __shfl_sync(0xffffffffu, rpart, rr);
            if (rr < nrows && okc) P.C[rp + cpart] = sg * stg[rr * (Cfg::CW + 1) + lane];
          }
        }
        __syncwarp();
      }
      if (nk > 0) {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[acc]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, Cfg::TMEM_COLS);
  }
}

// ---- host side -------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  // resolved once; static initialisation is thread-safe
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return nullptr;
  }();
  return fn;
}

// fmt: 0 = FP16, 1 = BF16, 2 = TF32 (FP32 words)
static bool encode_2d(CUtensorMap* m, const void* base, int fmt, int64_t rows, int32_t kdim, int32_t ldk,
                      int box_k, int box_rows) {
  auto enc = get_encode();
  if (!enc) return false;
  const CUtensorMapDataType ty = fmt == 0   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                 : fmt == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                            : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  cuuint64_t dims[2] = {(cuuint64_t)kdim, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ldk * (fmt == 2 ? 4 : 2)};
  cuuint32_t box[2] = {(cuuint32_t)box_k, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, ty, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// The four maps (A hi, B hi, A lo, B lo) of fused-matrix pair pi.
template <int FMT, bool SPLIT, int BN>
static bool encode_set(const TcOperands& ops, int pi, CUtensorMap* a_hi, CUtensorMap* b_hi, CUtensorMap* a_lo,
                       CUtensorMap* b_lo) {
  using Cfg = TcCfg<FMT, SPLIT, BN>;
  bool ok = encode_2d(a_hi, ops.a_hi[pi], FMT, ops.a_rows[pi], ops.kdim[pi], ops.ldk[pi], Cfg::KB, TC_BM) &&
            encode_2d(b_hi, ops.b_hi[pi], FMT, ops.b_rows[pi], ops.kdim[pi], ops.ldk[pi], Cfg::KB, BN);
  if (SPLIT)
    ok = ok && encode_2d(a_lo, ops.a_lo[pi], FMT, ops.a_rows[pi], ops.kdim[pi], ops.ldk[pi], Cfg::KB, TC_BM) &&
         encode_2d(b_lo, ops.b_lo[pi], FMT, ops.b_rows[pi], ops.kdim[pi], ops.ldk[pi], Cfg::KB, BN);
  return ok;
}

template <int FMT, bool SPLIT, int BN>
static ftn_status run(ftn_ctx ctx, const TcOperands* ops, const void* gmaps, const GemmProb* d_probs, int nprobs,
                      int64_t tiles, float* c, const TileEnt* tt) {
  using Cfg = TcCfg<FMT, SPLIT, BN>;
  TcParams P;
  std::memset(&P, 0, sizeof(P));
  for (int pi = 0; ops && pi < 2; ++pi) {
    if (ops->a_rows[pi] <= 0 || ops->b_rows[pi] <= 0 || ops->kdim[pi] <= 0) continue;
    if (!encode_set<FMT, SPLIT, BN>(*ops, pi, &P.a_hi[pi], &P.b_hi[pi], &P.a_lo[pi], &P.b_lo[pi]))
      return set_error(FTN_ECUDA, "cuTensorMapEncodeTiled failed");
  }
  P.gmaps = reinterpret_cast<const CUtensorMap*>(gmaps);
  P.tt = tt;
  P.probs = d_probs;
  P.C = c;
  P.err = ctx->dev_err;
  P.tiles = tiles;
  P.nprobs = nprobs;
  static const cudaError_t attr = cudaFuncSetAttribute(tc_gemm_kernel<FMT, SPLIT, BN>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
  if (attr != cudaSuccess) return cuda_error(attr, "cudaFuncSetAttribute(tc_gemm)");
  int64_t grid = tiles < ctx->num_sms ? tiles : ctx->num_sms;
  P.contig = tiles >= 8 * grid ? 1 : 0;
  cudaError_t e = launch_pdl(tc_gemm_kernel<FMT, SPLIT, BN>, (unsigned)grid, TC_THREADS, Cfg::SMEM, ctx->stream, P);
  ctx->launches += 1;
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "tc_gemm_kernel launch");
  return FTN_OK;
}

int tc_pick_bn(int max_n, ftn_prec prec) {
  const bool split = prec_split(prec);
  const int cap = split ? 128 : 256;
  int bn = 16;
  while (bn < max_n && bn < cap) bn *= 2;
  return bn;
}

int64_t tc_tiles_for(int M, int N, int bn) {
  return (int64_t)((M + TC_BM - 1) / TC_BM) * ((N + bn - 1) / bn);
}

template <int FMT, bool SPLIT>
static ftn_status by_bn(ftn_ctx ctx, int bn, const TcOperands* ops, const void* gm, const GemmProb* d, int np,
                        int64_t tiles, float* c, const TileEnt* tt) {
  switch (bn) {
    case 16: return run<FMT, SPLIT, 16>(ctx, ops, gm, d, np, tiles, c, tt);
    case 32: return run<FMT, SPLIT, 32>(ctx, ops, gm, d, np, tiles, c, tt);
    case 64: return run<FMT, SPLIT, 64>(ctx, ops, gm, d, np, tiles, c, tt);
    case 128: return run<FMT, SPLIT, 128>(ctx, ops, gm, d, np, tiles, c, tt);
    default:
      if constexpr (!SPLIT) return run<FMT, SPLIT, 256>(ctx, ops, gm, d, np, tiles, c, tt);
      return set_error(FTN_EINVAL, "bad tile width");
  }
}

static ftn_status dispatch(ftn_ctx ctx, ftn_prec prec, int bn, const TcOperands* ops, const void* gm,
                           const GemmProb* d_probs, int nprobs, int64_t tiles, float* c, const TileEnt* tt) {
  if (nprobs == 0 || tiles == 0) return FTN_OK;
  switch (prec) {
    case FTN_PREC_TF32: return by_bn<2, false>(ctx, bn, ops, gm, d_probs, nprobs, tiles, c, tt);
    case FTN_PREC_TF32X3: return by_bn<2, true>(ctx, bn, ops, gm, d_probs, nprobs, tiles, c, tt);
    case FTN_PREC_BF16: return by_bn<1, false>(ctx, bn, ops, gm, d_probs, nprobs, tiles, c, tt);
    case FTN_PREC_BF16X3: return by_bn<1, true>(ctx, bn, ops, gm, d_probs, nprobs, tiles, c, tt);
    case FTN_PREC_F16X3: return by_bn<0, true>(ctx, bn, ops, gm, d_probs, nprobs, tiles, c, tt);
    default: return set_error(FTN_EUNSUPPORTED, "precision has no tensor-core path");
  }
}

ftn_status launch_gemm_tc(ftn_ctx ctx, ftn_prec prec, const TcOperands& ops, const GemmProb* d_probs, int nprobs,
                          int64_t tiles, int bn, float* c, const TileEnt* tt) {
  return dispatch(ctx, prec, bn, &ops, nullptr, d_probs, nprobs, tiles, c, tt);
}

ftn_status tc_tile_table(ftn_ctx ctx, const GemmProb* d_probs, int nprobs, int64_t tiles, int bn, TileEnt* d_out) {
  if (tiles <= 0 || nprobs <= 0) return FTN_OK;
  TcParams P;
  std::memset(&P, 0, sizeof(P));
  P.probs = d_probs;
  P.nprobs = nprobs;
  P.tiles = tiles;
  const unsigned grid = (unsigned)std::min<int64_t>((tiles + 255) / 256, (int64_t)ctx->num_sms * 4);
  switch (bn) {
    case 16: tile_table_kernel<16><<<grid, 256, 0, ctx->stream>>>(P, d_out); break;
    case 32: tile_table_kernel<32><<<grid, 256, 0, ctx->stream>>>(P, d_out); break;
    case 64: tile_table_kernel<64><<<grid, 256, 0, ctx->stream>>>(P, d_out); break;
    case 128: tile_table_kernel<128><<<grid, 256, 0, ctx->stream>>>(P, d_out); break;
    case 256: tile_table_kernel<256><<<grid, 256, 0, ctx->stream>>>(P, d_out); break;
    default: return set_error(FTN_EINVAL, "bad tile width");
  }
  ctx->launches += 1;
  FTN_CUDA(cudaGetLastError());
  return FTN_OK;
}

ftn_status launch_gemm_tc_maps(ftn_ctx ctx, ftn_prec prec, const TcMapSet* d_maps, const GemmProb* d_probs,
                               int nprobs, int64_t tiles, int bn, float* c) {
  if (!d_maps || ((uintptr_t)d_maps & 63)) return set_error(FTN_EINVAL, "internal error: tensor maps not 64-byte aligned");
  return dispatch(ctx, prec, bn, nullptr, d_maps, d_probs, nprobs, tiles, c, nullptr);
}

template <int FMT, bool SPLIT>
static bool enc_by_bn(int bn, const TcOperands& ops, int pi, TcMapSet* out) {
  CUtensorMap* m = reinterpret_cast<CUtensorMap*>(out);
  switch (bn) {
    case 16: return encode_set<FMT, SPLIT, 16>(ops, pi, m, m + 1, m + 2, m + 3);
    case 32: return encode_set<FMT, SPLIT, 32>(ops, pi, m, m + 1, m + 2, m + 3);
    case 64: return encode_set<FMT, SPLIT, 64>(ops, pi, m, m + 1, m + 2, m + 3);
    case 128: return encode_set<FMT, SPLIT, 128>(ops, pi, m, m + 1, m + 2, m + 3);
    case 256: return !SPLIT && encode_set<FMT, SPLIT, 256>(ops, pi, m, m + 1, m + 2, m + 3);
    default: return false;
  }
}

ftn_status tc_encode_set(ftn_prec prec, int bn, const TcOperands& ops, int pi, TcMapSet* out) {
  static_assert(sizeof(TcMapSet) == 4 * sizeof(CUtensorMap), "map set layout");
  std::memset(out, 0, sizeof(TcMapSet));
  if (ops.a_rows[pi] <= 0 || ops.b_rows[pi] <= 0 || ops.kdim[pi] <= 0) return FTN_OK;
  bool ok = false;
  switch (prec) {
    case FTN_PREC_TF32: ok = enc_by_bn<2, false>(bn, ops, pi, out); break;
    case FTN_PREC_TF32X3: ok = enc_by_bn<2, true>(bn, ops, pi, out); break;
    case FTN_PREC_BF16: ok = enc_by_bn<1, false>(bn, ops, pi, out); break;
    case FTN_PREC_BF16X3: ok = enc_by_bn<1, true>(bn, ops, pi, out); break;
    case FTN_PREC_F16X3: ok = enc_by_bn<0, true>(bn, ops, pi, out); break;
    default: return set_error(FTN_EUNSUPPORTED, "precision has no tensor-core path");
  }
  return ok ? FTN_OK : set_error(FTN_ECUDA, "cuTensorMapEncodeTiled failed");
}

}  // namespace ftn
