// Fermionic tensordot (Eq. standardcontract with the bond parity of the
// locally ordered formalism, Eq. fermionictn2) and fermionic transposition
// (Eq. transposition): block-pair planning, per-block signs and the fused
// sector-matrix layout of Sec. IV.A, then sign-permute + grouped GEMM.
#include <algorithm>
#include <mutex>

#include "tdplan.h"

namespace ftn {

// parity (0/1) of the number of inverted pairs of set bits: out position u
// holds source leg perm[u]; bits are indexed by source leg.
int inversion_parity(int r, const int* perm, uint32_t mask) {
  int s = 0;
  for (int u = 0; u < r; ++u) {
    if (!((mask >> perm[u]) & 1)) continue;
    for (int v = u + 1; v < r; ++v)
      if (perm[u] > perm[v] && ((mask >> perm[v]) & 1)) s ^= 1;
  }
  return s;
}

uint32_t gather_bits(uint32_t mask, const int* legs, int n) {
  uint32_t m = 0;
  for (int i = 0; i < n; ++i) m |= ((mask >> legs[i]) & 1u) << i;
  return m;
}

// enumerate masks over `n` bits with a given parity, increasing order;
// returns cumulative offsets indexed by mask (size 2^n) and the total.
int64_t sector_offsets(int n, const int64_t* d0, const int64_t* d1, int parity, std::vector<int64_t>& off,
                       std::vector<int64_t>& size) {
  off.assign((size_t)1 << n, -1);
  size.assign((size_t)1 << n, 0);
  int64_t tot = 0;
  for (uint32_t m = 0; m < (1u << n); ++m) {
    if ((popc(m) & 1) != parity) continue;
    int64_t s = 1;
    for (int i = 0; i < n; ++i) s *= ((m >> i) & 1) ? d1[i] : d0[i];
    off[m] = tot;
    size[m] = s;
    tot += s;
  }
  return tot;
}

// Every index a permute job or a GEMM problem can touch must lie inside its
// buffers; a plan that fails this is rejected before any launch.
bool jobs_in_bounds(const std::vector<PermJob>& jobs, int64_t src_n, int64_t dst_n) {
  for (const PermJob& j : jobs) {
    int64_t ms = j.src_off, md = j.dst_off;
    const int nl = j.nI + j.nO + j.nB;
    for (int q = 0; q < nl; ++q) {
      if (j.dim[q] <= 0) return false;
      ms += (int64_t)(j.dim[q] - 1) * j.sstr[q];
      md += (int64_t)(j.dim[q] - 1) * j.dstr[q];
    }
    if (j.src_off < 0 || j.dst_off < 0 || ms >= src_n || md >= dst_n) return false;
    // the kernel keeps offsets relative to a block in 32-bit integers
    if (ms - j.src_off >= ((int64_t)1 << 31) || md - j.dst_off >= ((int64_t)1 << 31)) return false;
  }
  return true;
}

bool probs_in_bounds(const std::vector<GemmProb>& probs, int64_t a_n, int64_t b_n, int64_t c_n) {
  for (const GemmProb& g : probs) {
    if (g.M <= 0 || g.N <= 0 || g.K < 0) return false;
    if (g.K > 0) {
      if (g.a_off + (int64_t)(g.M - 1) * g.a_sm + (int64_t)(g.K - 1) * g.a_sk >= a_n) return false;
      if (g.b_off + (int64_t)(g.N - 1) * g.b_sn + (int64_t)(g.K - 1) * g.b_sk >= b_n) return false;
    }
    int64_t mr = 1, mc = 1, top = g.c_off + (g.nsplit > 1 ? (int64_t)(g.nsplit - 1) * g.c_slab : 0);
    if (g.nsplit > 1 && ((int64_t)g.nsplit * g.kchunk < g.K || g.kchunk <= 0)) return false;
    for (int l = 0; l < g.nrl; ++l) mr *= g.rdim[l], top += (int64_t)(g.rdim[l] - 1) * g.rstr[l];
    for (int l = 0; l < g.ncl; ++l) mc *= g.cdim[l], top += (int64_t)(g.cdim[l] - 1) * g.cstr[l];
    if (mr != g.M || mc != g.N || g.c_off < 0 || top >= c_n) return false;
  }
  return true;
}

static ftn_status upload_plan(ftn_ctx ctx, TdPlan& P) {
  size_t sa = P.ja.size() * sizeof(PermJob), sb = P.jb.size() * sizeof(PermJob), sc = P.jc.size() * sizeof(PermJob),
         sp = P.probs.size() * sizeof(GemmProb), sr = P.red.size() * sizeof(GemmProb),
         sm = P.jab.size() * sizeof(PermJob), sw = P.witems.size() * sizeof(WarpItem);
  const size_t pre = (sa + sb + sc + sp + sr + sm + sw + 255) & ~(size_t)255;
  const size_t st = P.tile_tab ? (size_t)P.gemm_tiles * sizeof(TileEnt) : 0;
  size_t tot = sa + sb + sc + sp + sr + sm + sw;
  std::vector<uint8_t> host(tot + 16);
  std::memcpy(host.data(), P.ja.data(), sa);
  std::memcpy(host.data() + sa, P.jb.data(), sb);
  std::memcpy(host.data() + sa + sb, P.jc.data(), sc);
  std::memcpy(host.data() + sa + sb + sc, P.probs.data(), sp);
  if (sr) std::memcpy(host.data() + sa + sb + sc + sp, P.red.data(), sr);
  if (sm) std::memcpy(host.data() + sa + sb + sc + sp + sr, P.jab.data(), sm);
  if (sw) std::memcpy(host.data() + sa + sb + sc + sp + sr + sm, P.witems.data(), sw);
  P.dev = std::make_shared<DevTables>();
  P.dev->ctx = ctx;
  void* d = nullptr;
  // (a pageable host-to-device copy has staged its source when the call returns)
  if (st) {  // room after the tables for the tile table, filled on the device below
    d = dev_alloc(ctx, pre + st);
    if (!d) return set_error(FTN_ENOMEM, "device allocation failed (plan tables)");
    FTN_CUDA(cudaMemcpyAsync(d, host.data(), tot, cudaMemcpyHostToDevice, ctx->stream));
  } else {
    FTN_TRY(upload_table(ctx, host.data(), tot, &d));
  }
  P.dev->p = d;
  uint8_t* b = (uint8_t*)d;
  P.d_ja = (PermJob*)b;
  P.d_jb = (PermJob*)(b + sa);
  P.d_jc = (PermJob*)(b + sa + sb);
  P.d_probs = (GemmProb*)(b + sa + sb + sc);
  P.d_red = sr ? (GemmProb*)(b + sa + sb + sc + sp) : nullptr;
  P.d_jab = sm ? (PermJob*)(b + sa + sb + sc + sp + sr) : nullptr;
  P.d_witems = sw ? (WarpItem*)(b + sa + sb + sc + sp + sr + sm) : nullptr;
  if (st) {
    P.d_tt = (TileEnt*)(b + pre);
    FTN_TRY(tc_tile_table(ctx, P.d_probs, P.n_tiled, P.gemm_tiles, P.bn, P.d_tt));
  }
  return FTN_OK;
}

// Plan caches are per context.  The maps from context to cache are shared
// by all host threads, so lookups and erasures take a lock; a cache itself
// is used only by the thread that drives its context (one host thread per
// context at a time), and std::map nodes do not move on insertion.
static std::mutex g_cache_mu;

static std::unordered_map<std::string, std::shared_ptr<TdPlan>>& plan_cache(ftn_ctx ctx) {
  static std::map<ftn_ctx, std::unordered_map<std::string, std::shared_ptr<TdPlan>>> caches;
  std::lock_guard<std::mutex> lock(g_cache_mu);
  return caches[ctx];
}

// bn_cap > 0 caps the tensor-core tile width (the tuner's candidates).
static ftn_status build_plan(ftn_ctx ctx, const ftn_tensor_s* A, const ftn_tensor_s* B, int n, const int* ax,
                             const int* ay, uint64_t flip_a, uint64_t flip_b, const int* out_perm, ftn_prec prec,
                             std::shared_ptr<TdPlan>& out, int bn_cap = 0) {
  auto P = std::make_shared<TdPlan>();
  P->n = n;
  bool in_a[MAXR] = {}, in_b[MAXR] = {};
  for (int i = 0; i < n; ++i) {
    in_a[ax[i]] = true;
    in_b[ay[i]] = true;
  }
  for (int k = 0; k < A->rank; ++k)
    if (!in_a[k]) P->fa[P->nfa++] = k;
  for (int k = 0; k < B->rank; ++k)
    if (!in_b[k]) P->fb[P->nfb++] = k;
  // Order of the free legs inside the fused matrices (any order gives the
  // same result: every sign is computed from the orders actually used).
  // With an output permutation each side's free legs go in the order of
  // their destination positions, the fastest last, so that the epilogue's
  // write runs follow the GEMM row or column index.  gidx maps a result leg
  // (A's free legs, then B's, in leg order) to its position in that order.
  int gidx[MAXR];
  for (int r = 0; r < P->nfa + P->nfb; ++r) gidx[r] = r;
  if (out_perm) {
    const int cr_api = P->nfa + P->nfb;
    int outpos[MAXR];
    for (int u = 0; u < cr_api; ++u) outpos[out_perm[u]] = u;
    int oa[MAXR], ob[MAXR];
    for (int j = 0; j < P->nfa; ++j) oa[j] = j;
    for (int j = 0; j < P->nfb; ++j) ob[j] = P->nfa + j;
    std::stable_sort(oa, oa + P->nfa, [&](int x, int y) { return outpos[x] < outpos[y]; });
    std::stable_sort(ob, ob + P->nfb, [&](int x, int y) { return outpos[x] < outpos[y]; });
    int fa_api[MAXR], fb_api[MAXR];
    for (int j = 0; j < P->nfa; ++j) fa_api[j] = P->fa[j];
    for (int j = 0; j < P->nfb; ++j) fb_api[j] = P->fb[j];
    for (int i = 0; i < P->nfa; ++i) {
      P->fa[i] = fa_api[oa[i]];
      gidx[oa[i]] = i;
    }
    for (int i = 0; i < P->nfb; ++i) {
      P->fb[i] = fb_api[ob[i] - P->nfa];
      gidx[ob[i]] = P->nfa + i;
    }
  }
  const int pA = A->parity, pB = B->parity;
  // sector offsets of free rows (A), free columns (B) and the fused bond (K)
  int64_t fad0[MAXR], fad1[MAXR], fbd0[MAXR], fbd1[MAXR], kd0[MAXR], kd1[MAXR];
  for (int j = 0; j < P->nfa; ++j) fad0[j] = A->d0[P->fa[j]], fad1[j] = A->d1[P->fa[j]];
  for (int j = 0; j < P->nfb; ++j) fbd0[j] = B->d0[P->fb[j]], fbd1[j] = B->d1[P->fb[j]];
  for (int i = 0; i < n; ++i) kd0[i] = A->d0[ax[i]], kd1[i] = A->d1[ax[i]];
  std::vector<int64_t>*rowoff = P->rowoff, *rowsz = P->rowsz, *coloff = P->coloff, *colsz = P->colsz;
  std::vector<int64_t> koff[2], ksz[2];
  for (int pi = 0; pi < 2; ++pi) {
    P->M[pi] = sector_offsets(P->nfa, fad0, fad1, pA ^ pi, rowoff[pi], rowsz[pi]);
    P->N[pi] = sector_offsets(P->nfb, fbd0, fbd1, pB ^ pi, coloff[pi], colsz[pi]);
    P->K[pi] = sector_offsets(n, kd0, kd1, pi, koff[pi], ksz[pi]);
    P->ldk[pi] = std::max<int64_t>(8, (P->K[pi] + 7) / 8 * 8);
  }
  P->afoff[0] = 0;
  P->afoff[1] = (P->M[0] * P->ldk[0] + 63) / 64 * 64;
  P->af_elems = P->afoff[1] + P->M[1] * P->ldk[1];
  P->bfoff[0] = 0;
  P->bfoff[1] = (P->N[0] * P->ldk[0] + 63) / 64 * 64;
  P->bf_elems = P->bfoff[1] + P->N[1] * P->ldk[1];

  // ---- A blocks -> fused A_pi rows ----
  int permA[MAXR], permB[MAXR];
  for (int j = 0; j < P->nfa; ++j) permA[j] = P->fa[j];
  for (int i = 0; i < n; ++i) permA[P->nfa + i] = ax[i];
  for (int i = 0; i < n; ++i) permB[i] = ay[n - 1 - i];
  for (int j = 0; j < P->nfb; ++j) permB[n + j] = P->fb[j];
  uint32_t arrow_a = 0;
  for (int i = 0; i < n; ++i)
    if (A->dual[ax[i]] == 0) arrow_a |= 1u << ax[i];
  for (int64_t b = 0; b < nblocks(A->rank, pA); ++b) {
    uint32_t m = block_mask(A->rank, pA, b);
    uint32_t mA = gather_bits(m, P->fa, P->nfa), mK = gather_bits(m, ax, n);
    int pi = popc(mK) & 1;
    int64_t dims[MAXR], dstr[MAXR];
    for (int k = 0; k < A->rank; ++k) dims[k] = leg_dim(A, k, m);
    int64_t s = P->ldk[pi];
    for (int j = P->nfa - 1; j >= 0; --j) {
      dstr[P->fa[j]] = s;
      s *= dims[P->fa[j]];
    }
    s = 1;
    for (int i = n - 1; i >= 0; --i) {
      dstr[ax[i]] = s;
      s *= dims[ax[i]];
    }
    int sg = inversion_parity(A->rank, permA, m) ^ (popc(m & arrow_a) & 1) ^ (popc(m & (uint32_t)flip_a) & 1);
    int64_t dst = P->afoff[pi] + rowoff[pi][mA] * P->ldk[pi] + koff[pi][mK];
    add_perm_job(P->ja, P->ta, A->rank, dims, dstr, A->offsets[b], dst, sg ? -1 : 1);
  }
  // ---- B blocks -> fused B_pi^T rows (K-major) ----
  for (int64_t b = 0; b < nblocks(B->rank, pB); ++b) {
    uint32_t m = block_mask(B->rank, pB, b);
    uint32_t mB = gather_bits(m, P->fb, P->nfb), mK = gather_bits(m, ay, n);
    int pi = popc(mK) & 1;
    int64_t dims[MAXR], dstr[MAXR];
    for (int k = 0; k < B->rank; ++k) dims[k] = leg_dim(B, k, m);
    int64_t s = P->ldk[pi];
    for (int j = P->nfb - 1; j >= 0; --j) {
      dstr[P->fb[j]] = s;
      s *= dims[P->fb[j]];
    }
    s = 1;
    for (int i = n - 1; i >= 0; --i) {
      dstr[ay[i]] = s;
      s *= dims[ay[i]];
    }
    int sg = inversion_parity(B->rank, permB, m) ^ (popc(m & (uint32_t)flip_b) & 1);
    int64_t dst = P->bfoff[pi] + coloff[pi][mB] * P->ldk[pi] + koff[pi][mK];
    add_perm_job(P->jb, P->tb, B->rank, dims, dstr, B->offsets[b], dst, sg ? -1 : 1);
  }
  // the staged permute needs 16-byte aligned source rows (buffer base included)
  const bool al_a = ((uintptr_t)A->data & 15) == 0, al_b = ((uintptr_t)B->data & 15) == 0;
  std::vector<PermJob> ja_raw = P->ja, jb_raw = P->jb;
  P->sa = finalize_perm_jobs(P->ja, dtype_size(A->dtype), &P->ta, al_a);
  P->sb = finalize_perm_jobs(P->jb, dtype_size(B->dtype), &P->tb, al_b);
  // Both operands in one launch: B's jobs read the second source and write
  // after A's fused matrices (the workspace holds [A hi | B hi | A lo | B lo]).
  // Kept when the merged list runs on the shared-memory-staged kernel, or when both
  // operands were on the register-staged one anyway.
  if (!ja_raw.empty() && !jb_raw.empty()) {
    const bool half = prec_half(prec);
    const int64_t es_out = prec == FTN_PREC_F64 ? 8 : (half ? 2 : 4);
    const int64_t a_bytes = ((int64_t)P->af_elems * es_out + 255) / 256 * 256;
    std::vector<PermJob> m = ja_raw;
    for (PermJob j : jb_raw) {
      j.src_sel = 1;
      j.dst_off += a_bytes / es_out;
      m.push_back(j);
    }
    int64_t t = 0;
    const int st = finalize_perm_jobs(m, dtype_size(A->dtype), &t, al_a && al_b);
    if (st || (!P->sa && !P->sb)) {
      P->jab = std::move(m);
      P->tab = t;
      P->sab = st;
    }
  }
  // ---- result metadata (before out_perm) ----
  const int cr = P->nfa + P->nfb;
  ftn_tensor_s tmp;
  tmp.rank = cr;
  tmp.parity = pA ^ pB;
  for (int j = 0; j < P->nfa; ++j) {
    tmp.d0[j] = A->d0[P->fa[j]];
    tmp.d1[j] = A->d1[P->fa[j]];
    tmp.dual[j] = A->dual[P->fa[j]];
  }
  for (int j = 0; j < P->nfb; ++j) {
    tmp.d0[P->nfa + j] = B->d0[P->fb[j]];
    tmp.d1[P->nfa + j] = B->d1[P->fb[j]];
    tmp.dual[P->nfa + j] = B->dual[P->fb[j]];
  }
  std::vector<int64_t> toff(nblocks(cr, tmp.parity));
  int64_t tot = 0;
  for (int64_t b = 0; b < (int64_t)toff.size(); ++b) {
    toff[b] = tot;
    tot += block_size(&tmp, block_mask(cr, tmp.parity, b));
  }
  P->tmp_numel = tot;
  // ---- final result layout (out_perm applied in the GEMM epilogue) ----
  P->cr = cr;
  P->cpar = tmp.parity;
  // output leg u = leg perm[u] of the GEMM-order result
  int perm[MAXR];
  for (int u = 0; u < cr; ++u) perm[u] = gidx[out_perm ? out_perm[u] : u];
  bool ident = true;
  for (int u = 0; u < cr; ++u) ident = ident && perm[u] == u;
  P->out_perm = !ident;
  for (int u = 0; u < cr; ++u)
    P->cd0[u] = tmp.d0[perm[u]], P->cd1[u] = tmp.d1[perm[u]], P->cdual[u] = tmp.dual[perm[u]];
  ftn_tensor_s fin;
  fin.rank = cr;
  fin.parity = tmp.parity;
  for (int u = 0; u < cr; ++u) fin.d0[u] = P->cd0[u], fin.d1[u] = P->cd1[u];
  std::vector<int64_t> foff(nblocks(cr, fin.parity));
  int64_t fin_numel = 0;
  for (int64_t b = 0; b < (int64_t)foff.size(); ++b) {
    foff[b] = fin_numel;
    fin_numel += block_size(&fin, block_mask(cr, fin.parity, b));
  }
  P->tmp_numel = fin_numel;
  // ---- how the result reaches its final layout ----
  // The epilogue writes 32 consecutive columns (or rows) per warp store; it
  // applies the permutation itself when the destination's fastest legs form
  // a long enough run along one of those directions, otherwise the GEMM
  // writes the plain block layout and a sign-permute pass follows.
  bool fuse = true;
  int epi_rows = 0;
  if (P->out_perm) {
    int64_t run_c = 1, run_r = 1;
    for (int u = cr - 1, k = cr - 1; u >= 0 && k >= P->nfa && perm[u] == k; --u, --k)
      run_c *= std::max(1, std::min(tmp.d0[k] ? tmp.d0[k] : tmp.d1[k], tmp.d1[k] ? tmp.d1[k] : tmp.d0[k]));
    for (int u = cr - 1, k = P->nfa - 1; u >= 0 && k >= 0 && perm[u] == k; --u, --k)
      run_r *= std::max(1, std::min(tmp.d0[k] ? tmp.d0[k] : tmp.d1[k], tmp.d1[k] ? tmp.d1[k] : tmp.d0[k]));
    if (run_c >= 16 && run_c >= run_r) {
      epi_rows = 0;
    } else if (run_r >= 16) {
      epi_rows = 1;
    } else if (fin_numel <= ((int64_t)1 << 22)) {
      // short runs, small result: scattered epilogue stores cost less than a
      // second pass over the result
      epi_rows = run_r > run_c ? 1 : 0;
    } else {
      fuse = false;
    }
  }
  P->fused = fuse;
  if (!fuse) P->tmp_numel = tot;
  // ---- GEMM problems, one per result block ----
  const bool tc = prec != FTN_PREC_F64;
  int maxN = 1;
  for (int64_t b = 0; b < (int64_t)toff.size(); ++b) {
    uint32_t m = block_mask(cr, tmp.parity, b);
    uint32_t mB = m >> P->nfa;
    int pi = (popc(mB) & 1) ^ pB;
    maxN = std::max<int64_t>(maxN, colsz[pi][mB]);
  }
  P->bn = tc ? tc_pick_bn(maxN, prec) : f64_pick_bn(maxN);
  if (tc && bn_cap > 0) P->bn = std::min(P->bn, bn_cap);
  for (int64_t b = 0; b < (int64_t)toff.size(); ++b) {
    uint32_t m = block_mask(cr, tmp.parity, b);
    uint32_t mA = m & ((1u << P->nfa) - 1u), mB = m >> P->nfa;
    int pi = (popc(mA) & 1) ^ pA;
    GemmProb g;
    std::memset(&g, 0, sizeof(g));
    g.M = (int32_t)rowsz[pi][mA];
    g.N = (int32_t)colsz[pi][mB];
    g.K = (int32_t)P->K[pi];
    if (g.M == 0 || g.N == 0) continue;
    g.pi = pi;
    g.lda = g.ldb = (int32_t)P->ldk[pi];
    g.a_row0 = (int32_t)rowoff[pi][mA];
    g.b_row0 = (int32_t)coloff[pi][mB];
    g.a_off = P->afoff[pi] + rowoff[pi][mA] * P->ldk[pi];
    g.b_off = P->bfoff[pi] + coloff[pi][mB] * P->ldk[pi];
    g.a_sm = g.b_sn = P->ldk[pi];
    g.a_sk = g.b_sk = 1;
    if (fuse) {
      // destination block in the (permuted) result and the stride of each leg
      uint32_t mo = 0;
      for (int u = 0; u < cr; ++u) mo |= ((m >> perm[u]) & 1u) << u;
      int64_t dims[MAXR], str[MAXR];
      for (int k = 0; k < cr; ++k) dims[k] = leg_dim(&tmp, k, m);
      int64_t st = 1;
      for (int u = cr - 1; u >= 0; --u) {
        str[perm[u]] = st;
        st *= dims[perm[u]];
      }
      g.c_off = cr == 0 ? 0 : foff[mo >> 1];
      g.c_sign = inversion_parity(cr, perm, m) ? -1 : 1;
      g.nrl = P->nfa;
      g.ncl = P->nfb;
      for (int k = 0; k < P->nfa; ++k) g.rdim[k] = (int32_t)dims[k], g.rstr[k] = str[k];
      for (int k = 0; k < P->nfb; ++k) g.cdim[k] = (int32_t)dims[P->nfa + k], g.cstr[k] = str[P->nfa + k];
      g.epi_rows = epi_rows;
    } else {
      // plain row-major block of the unpermuted result
      g.c_off = toff[b];
      g.c_sign = 1;
      g.nrl = g.ncl = 1;
      g.rdim[0] = g.M;
      g.rstr[0] = g.N;
      g.cdim[0] = g.N;
      g.cstr[0] = 1;
    }
    if (tc) {
      g.tiles_m = (g.M + 127) / 128;
      g.tiles_n = (g.N + P->bn - 1) / P->bn;
    } else {
      g.tiles_m = (g.M + 63) / 64;
      g.tiles_n = (g.N + P->bn - 1) / P->bn;
    }
    P->probs.push_back(g);
  }
  // vector stores in the epilogue: the fastest leg along the write direction
  // has stride 1 and a dimension divisible by 4; every other stride and the
  // block offset are multiples of 4 elements
  for (GemmProb& g : P->probs) {
    bool ok = g.c_off % 4 == 0;
    const int nf = g.epi_rows ? g.nrl : g.ncl;
    const int32_t* fd = g.epi_rows ? g.rdim : g.cdim;
    const int64_t* fs = g.epi_rows ? g.rstr : g.cstr;
    ok = ok && nf > 0 && fs[nf - 1] == 1 && fd[nf - 1] % 4 == 0;
    for (int l = 0; l < g.nrl; ++l)
      if (!(g.epi_rows && l == nf - 1)) ok = ok && g.rstr[l] % 4 == 0;
    for (int l = 0; l < g.ncl; ++l)
      if (!(!g.epi_rows && l == nf - 1)) ok = ok && g.cstr[l] % 4 == 0;
    g.vec4 = ok ? 1 : 0;
  }
  // small tensor-core-precision problems run on CUDA cores (after the
  // grouped tile list, which covers probs[0, n_tiled))
  std::vector<GemmProb> small_tc;
  if (tc) {
    auto mid = std::stable_partition(P->probs.begin(), P->probs.end(), [](const GemmProb& g) { return !tcw_small(g); });
    small_tc.assign(mid, P->probs.end());
    P->probs.erase(mid, P->probs.end());
  }
  if (tc) {
    // group problems by (pi, row block); inside a group the tiles run
    // m-tile by m-tile across all member problems (A tile reuse in L2)
    std::stable_sort(P->probs.begin(), P->probs.end(), [](const GemmProb& x, const GemmProb& y) {
      if (x.pi != y.pi) return x.pi < y.pi;
      if (x.a_row0 != y.a_row0) return x.a_row0 < y.a_row0;
      return x.b_row0 < y.b_row0;
    });
    std::vector<std::pair<size_t, size_t>> groups;
    for (size_t i = 0; i < P->probs.size();) {
      size_t j = i;
      while (j < P->probs.size() && P->probs[j].pi == P->probs[i].pi && P->probs[j].a_row0 == P->probs[i].a_row0) ++j;
      groups.push_back({i, j});
      i = j;
    }
    // Merged groups: when every group's column blocks are adjacent rows of
    // B_pi and each a multiple of 32 wide, a tile may cross problems (its
    // epilogue picks the member per 32-column chunk), so the tile width
    // follows the group's total width: fewer, wider tiles and one read of
    // each A tile.
    bool merge = !groups.empty();
    int max_group_n = 1;
    for (auto& gr : groups) {
      int tot = 0;
      for (size_t q = gr.first; q < gr.second; ++q) {
        const GemmProb& g = P->probs[q];
        merge = merge && g.N % 32 == 0 && (q == gr.first || g.b_row0 == P->probs[q - 1].b_row0 + P->probs[q - 1].N);
        tot += g.N;
      }
      max_group_n = std::max(max_group_n, tot);
    }
    const int bn_merged = bn_cap > 0 ? std::min(tc_pick_bn(max_group_n, prec), bn_cap) : tc_pick_bn(max_group_n, prec);
    merge = merge && bn_merged > P->bn && bn_merged >= 32;
    if (merge) {  // only while the wider tiles still fill the GPU twice over
      int64_t mt = 0;
      for (auto& gr : groups) {
        int tot = 0;
        for (size_t q = gr.first; q < gr.second; ++q) tot += P->probs[q].N;
        mt += (int64_t)P->probs[gr.first].tiles_m * ((tot + bn_merged - 1) / bn_merged);
      }
      merge = mt >= 2 * (int64_t)ctx->num_sms;
    }
    if (merge) P->bn = bn_merged;
    for (auto& gr : groups) {
      int32_t row_tiles = 0, gcol = 0;
      for (size_t q = gr.first; q < gr.second; ++q) {
        GemmProb& g = P->probs[q];
        g.tiles_n = (g.N + P->bn - 1) / P->bn;
        g.tn_off = row_tiles;
        g.gmerge = merge ? 1 : 0;
        g.gcol = gcol;
        gcol += g.N;
        row_tiles += g.tiles_n;
      }
      if (merge) row_tiles = (gcol + P->bn - 1) / P->bn;
      for (size_t q = gr.first; q < gr.second; ++q) {
        GemmProb& g = P->probs[q];
        g.grp_first = (int32_t)gr.first;
        g.grp_count = (int32_t)(gr.second - gr.first);
        g.row_tiles = row_tiles;
        g.tile_begin = P->gemm_tiles;
      }
      P->gemm_tiles += (int64_t)P->probs[gr.first].tiles_m * row_tiles;
    }
    P->n_tiled = (int)P->probs.size();
    P->witems.clear();
    for (const GemmProb& g : small_tc) {
      f64w_items(g, (int)P->probs.size(), P->witems);
      P->probs.push_back(g);
    }
  } else {
    for (GemmProb& g : P->probs) {
      g.tile_begin = P->gemm_tiles;
      P->gemm_tiles += (int64_t)g.tiles_m * g.tiles_n;
    }
    P->part_elems = plan_splitk_f64(P->probs, ctx->num_sms, P->red, P->gemm_tiles, P->red_total);
    P->n_tiled = partition_f64(P->probs, P->witems, P->gemm_tiles);
  }
  // ---- the separate sign-permute of the result, when not fused ----
  if (!fuse) {
    for (int64_t b = 0; b < (int64_t)toff.size(); ++b) {
      uint32_t m = block_mask(cr, tmp.parity, b);
      uint32_t mo = 0;
      for (int u = 0; u < cr; ++u) mo |= ((m >> perm[u]) & 1u) << u;
      int64_t dims[MAXR], dstr[MAXR];
      for (int k = 0; k < cr; ++k) dims[k] = leg_dim(&tmp, k, m);
      int64_t st = 1;
      for (int u = cr - 1; u >= 0; --u) {
        dstr[perm[u]] = st;
        st *= dims[perm[u]];
      }
      int sg = inversion_parity(cr, perm, m);
      add_perm_job(P->jc, P->tc, cr, dims, dstr, toff[b], foff[mo >> 1], sg ? -1 : 1);
    }
    P->sc = finalize_perm_jobs(P->jc, dtype_size(A->dtype), &P->tc, true);
  }
  if (!jobs_in_bounds(P->ja, A->numel, P->af_elems) || !jobs_in_bounds(P->jb, B->numel, P->bf_elems) ||
      !probs_in_bounds(P->probs, P->af_elems, P->bf_elems, P->part_elems ? P->part_elems : P->tmp_numel) ||
      (P->part_elems && !red_in_bounds(P->red, P->part_elems, P->tmp_numel)) ||
      (!P->fused && !jobs_in_bounds(P->jc, P->tmp_numel, P->tmp_numel)))
    return set_error(FTN_EINVAL, "internal error: contraction plan out of bounds");
  // tensor-core launches read their tiles from a table decoded once here
  P->tile_tab = prec != FTN_PREC_F64 && P->gemm_tiles > 0 && P->gemm_tiles <= ((int64_t)1 << 20);
  FTN_TRY(upload_plan(ctx, *P));
  out = P;
  return FTN_OK;
}

ftn_status validate_pairs(const ftn_tensor_s* A, const ftn_tensor_s* B, int n, const int* ax, const int* ay) {
  if (n < 0 || n > A->rank || n > B->rank) return set_error(FTN_EINVAL, "bad number of contracted legs");
  if (n > 0 && (!ax || !ay)) return set_error(FTN_EINVAL, "null axes");
  bool ua[MAXR] = {}, ub[MAXR] = {};
  for (int i = 0; i < n; ++i) {
    if (ax[i] < 0 || ax[i] >= A->rank || ay[i] < 0 || ay[i] >= B->rank)
      return set_error(FTN_EINVAL, "axis out of range");
    if (ua[ax[i]] || ub[ay[i]]) return set_error(FTN_EINVAL, "repeated axis");
    ua[ax[i]] = ub[ay[i]] = true;
    if (A->d0[ax[i]] != B->d0[ay[i]] || A->d1[ax[i]] != B->d1[ay[i]])
      return set_error(FTN_ESHAPE, "contracted legs differ in sector dimensions");
    if (A->dual[ax[i]] == B->dual[ay[i]]) return set_error(FTN_EDUAL, "contracted legs must have opposite duals");
  }
  if (A->rank + B->rank - 2 * n > FTN_MAX_RANK) return set_error(FTN_EINVAL, "result rank exceeds FTN_MAX_RANK");
  return FTN_OK;
}

static std::string plan_key(const ftn_tensor_s* A, const ftn_tensor_s* B, int n, const int* ax, const int* ay,
                            uint64_t fa, uint64_t fb, const int* out_perm, ftn_prec prec) {
  CacheKey key;
  key.meta(A).meta(B).ints(ax, n).ints(ay, n).put(fa).put(fb).put<int32_t>((int32_t)prec);
  key.put<uint8_t>(((uintptr_t)A->data & 15) == 0).put<uint8_t>(((uintptr_t)B->data & 15) == 0);
  key.put<uint8_t>(out_perm != nullptr);
  if (out_perm) key.ints(out_perm, A->rank + B->rank - 2 * n);
  return key.s;
}

ftn_status get_plan(ftn_ctx ctx, const ftn_tensor_s* A, const ftn_tensor_s* B, int n, const int* ax,
                           const int* ay, uint64_t fa, uint64_t fb, const int* out_perm, ftn_prec prec,
                           std::shared_ptr<TdPlan>& P, bool* fresh) {
  const std::string key = plan_key(A, B, n, ax, ay, fa, fb, out_perm, prec);
  auto& cache = plan_cache(ctx);
  auto it = cache.find(key);
  if (it != cache.end()) {
    P = it->second;
    if (fresh) *fresh = false;
    return FTN_OK;
  }
  if (stream_capturing(ctx->stream))
    return set_error(FTN_EUNSUPPORTED, "a contraction's plan is not built while the stream is captured: run the "
                                       "contraction once before capturing it");
  FTN_TRY(build_plan(ctx, A, B, n, ax, ay, fa, fb, out_perm, prec, P));
  if (cache.size() > 65536) cache.clear();
  cache[key] = P;
  if (fresh) *fresh = true;
  return FTN_OK;
}

static ftn_status run_plan(ftn_ctx ctx, TdPlan& Pl, const ftn_tensor_s* A, const ftn_tensor_s* B, ftn_tensor out,
                          ftn_prec prec);
static ftn_status tune_plan(ftn_ctx ctx, const ftn_tensor_s* A, const ftn_tensor_s* B, int n, const int* ax,
                           const int* ay, uint64_t fa, uint64_t fb, const int* out_perm, ftn_prec prec,
                           std::shared_ptr<TdPlan>& P, ftn_tensor out);

ftn_status tensordot_impl(ftn_ctx ctx, ftn_tensor A, ftn_tensor B, int n, const int* ax, const int* ay,
                          uint64_t flip_a, uint64_t flip_b, const int* out_perm, ftn_prec prec, ftn_tensor* C) {
  if (!ctx || !A || !B || !C) return set_error(FTN_EINVAL, "null argument");
  if (A->dtype != B->dtype) return set_error(FTN_EINVAL, "A and B must have the same dtype");
  if ((prec == FTN_PREC_F64) != (A->dtype == FTN_F64))
    return set_error(FTN_EUNSUPPORTED, "FTN_PREC_F64 needs FP64 tensors; tensor-core precisions need FP32 tensors");
  if (!prec_valid(prec)) return set_error(FTN_EINVAL, "bad precision");
  FTN_TRY(validate_pairs(A, B, n, ax, ay));
  const int cr = A->rank + B->rank - 2 * n;
  if (out_perm) {
    bool seen[MAXR] = {};
    for (int u = 0; u < cr; ++u) {
      if (out_perm[u] < 0 || out_perm[u] >= cr || seen[out_perm[u]]) return set_error(FTN_EINVAL, "bad out_perm");
      seen[out_perm[u]] = true;
    }
  }
  std::shared_ptr<TdPlan> P;
  bool fresh = false;
  FTN_TRY(get_plan(ctx, A, B, n, ax, ay, flip_a, flip_b, out_perm, prec, P, &fresh));
  ftn_tensor out = *C;
  bool created = false;
  if (out) {
    if (!same_meta(out, cr, P->cd0, P->cd1, P->cdual, P->cpar, A->dtype))
      return set_error(FTN_EINVAL, "preallocated output has the wrong metadata");
    if ((uintptr_t)out->data & 15)  // the epilogues store 16-byte vectors
      return set_error(FTN_EINVAL, "preallocated output must be 16-byte aligned");
  } else {
    FTN_TRY(make_tensor(ctx, cr, P->cd0, P->cd1, P->cdual, P->cpar, A->dtype, &out));
    created = true;
  }
  ftn_status st = FTN_OK;
  if (fresh) st = tune_plan(ctx, A, B, n, ax, ay, flip_a, flip_b, out_perm, prec, P, out);
  if (st == FTN_OK) st = run_plan(ctx, *P, A, B, out, prec);
  if (st != FTN_OK) {
    if (created) ftn_tensor_free(out);
    return st;
  }
  *C = out;
  return FTN_OK;
}

// One contraction along plan P into `out` (asynchronous on the context's
// stream).
static ftn_status run_plan(ftn_ctx ctx, TdPlan& Pl, const ftn_tensor_s* A, const ftn_tensor_s* B, ftn_tensor out,
                          ftn_prec prec) {
  TdPlan* P = &Pl;
  // workspace: A_f (hi, lo), B_f (hi, lo), pre-permutation result
  const bool tc = prec != FTN_PREC_F64;
  const bool split = prec_split(prec);
  const bool bf16 = prec_half(prec);  // 16-bit operands
  const size_t es = tc ? (bf16 ? 2 : 4) : 8;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t a_b = al((size_t)P->af_elems * es), b_b = al((size_t)P->bf_elems * es);
  const size_t c_b = P->fused ? 0 : al((size_t)P->tmp_numel * dtype_size(A->dtype));
  const size_t p_b = al((size_t)P->part_elems * 8);
  const size_t need = a_b * (split ? 2 : 1) + b_b * (split ? 2 : 1) + c_b + p_b;
  uint8_t* ws = (uint8_t*)workspace(ctx, need);
  if (!ws) return set_error(FTN_ENOMEM, "workspace allocation failed");
  // [A hi | B hi | A lo | B lo]: both lo planes at one offset from their hi planes
  uint8_t* af_hi = ws;
  uint8_t* bf_hi = ws + a_b;
  uint8_t* af_lo = split ? ws + a_b + b_b : nullptr;
  uint8_t* bf_lo = split ? af_lo + a_b : nullptr;
  // the GEMM epilogue writes the final layout, or the plain one into workspace
  uint8_t* ctmp = P->fused ? (uint8_t*)out->data : ws + (a_b + b_b) * (split ? 2 : 1);
  const int mode = prec_perm_mode(prec);
  const double in_es = (double)dtype_size(A->dtype), planes = split ? 2.0 : 1.0;
  double gemm_flops = 0;
  for (const GemmProb& g : P->probs) gemm_flops += 2.0 * g.M * g.N * g.K;
  ftn_status st = FTN_OK;
  int rec = -1;
  const ftn_dtype in_type = A->dtype;
  if (P->d_jab) {  // both operands in one launch
    rec = prof_begin(ctx, "permute", (A->numel + B->numel) * (in_es + es * planes), 0);
    st = launch_permute2(ctx, P->d_jab, (int)P->jab.size(), P->tab, P->sab, A->data, B->data, af_hi, af_lo,
                         A->dtype, mode);
    prof_end(ctx, rec);
  } else {
    rec = prof_begin(ctx, "permute", A->numel * (in_es + es * planes), 0);
    st = launch_permute(ctx, P->d_ja, (int)P->ja.size(), P->ta, P->sa, A->data, af_hi, af_lo, A->dtype, mode);
    prof_end(ctx, rec);
    if (st == FTN_OK) {
      rec = prof_begin(ctx, "permute", B->numel * (in_es + es * planes), 0);
      st = launch_permute(ctx, P->d_jb, (int)P->jb.size(), P->tb, P->sb, B->data, bf_hi, bf_lo, B->dtype, mode);
      prof_end(ctx, rec);
    }
  }
  if (st == FTN_OK) {
    double gb = 0;
    for (int pi = 0; pi < 2; ++pi) gb += (double)(P->M[pi] + P->N[pi]) * P->K[pi] * es * planes;
    gb += (double)P->tmp_numel * in_es;
    if (!tc) {
      rec = prof_begin(ctx, "gemm_f64", gb, gemm_flops);
      double* dst = P->part_elems ? (double*)(ws + need - p_b) : (double*)ctmp;
      st = launch_gemm_f64(ctx, P->d_probs, P->n_tiled, P->gemm_tiles, (const double*)af_hi, (const double*)bf_hi, dst,
                           P->bn);
      if (st == FTN_OK)
        st = launch_gemm_f64_warp(ctx, P->d_probs, P->d_witems, (int)P->witems.size(), (const double*)af_hi,
                                  (const double*)bf_hi, dst);
      if (st == FTN_OK && P->part_elems)
        st = launch_splitk_reduce(ctx, P->d_red, (int)P->red.size(), P->red_total, dst, (double*)ctmp);
      prof_end(ctx, rec);
    } else {
      TcOperands ops;
      for (int pi = 0; pi < 2; ++pi) {
        ops.a_hi[pi] = af_hi + P->afoff[pi] * es;
        ops.b_hi[pi] = bf_hi + P->bfoff[pi] * es;
        ops.a_lo[pi] = split ? af_lo + P->afoff[pi] * es : nullptr;
        ops.b_lo[pi] = split ? bf_lo + P->bfoff[pi] * es : nullptr;
        ops.a_rows[pi] = P->M[pi];
        ops.b_rows[pi] = P->N[pi];
        ops.kdim[pi] = (int32_t)P->K[pi];
        ops.ldk[pi] = (int32_t)P->ldk[pi];
      }
      rec = prof_begin(ctx, "gemm_tc", gb, gemm_flops);
      st = launch_gemm_tc(ctx, prec, ops, P->d_probs, P->n_tiled, P->gemm_tiles, P->bn, (float*)ctmp, P->d_tt);
      if (st == FTN_OK)
        st = launch_gemm_f32_warp(ctx, prec, P->d_probs, P->d_witems, (int)P->witems.size(), af_hi, bf_hi,
                                  split ? (int64_t)((af_lo - af_hi) / (int64_t)es) : 0, (float*)ctmp);
      prof_end(ctx, rec);
    }
  }
  if (st == FTN_OK && !P->fused) {
    rec = prof_begin(ctx, "permute", 2.0 * P->tmp_numel * in_es, 0);
    st = launch_permute(ctx, P->d_jc, (int)P->jc.size(), P->tc, P->sc, ctmp, out->data, nullptr, in_type, PERM_SAME);
    prof_end(ctx, rec);
  }
  return st;
}

// Tile-width tuner.  On the first use of a tensor-core plan of at least
// 2^30 sector flops (outside stream capture) the same contraction is also
// planned with the GEMM tile width capped at half and a quarter of the
// default (at least 32), each candidate is run once to warm up and once
// under CUDA events, and the fastest is kept in the plan cache.  The tile
// width does not change any result bit: every output element accumulates
// its K products in the same order whatever the tiling.  `out` holds the
// contraction afterwards.
static ftn_status tune_plan(ftn_ctx ctx, const ftn_tensor_s* A, const ftn_tensor_s* B, int n, const int* ax,
                           const int* ay, uint64_t fa, uint64_t fb, const int* out_perm, ftn_prec prec,
                           std::shared_ptr<TdPlan>& P, ftn_tensor out) {
  if (!ctx->tune || prec == FTN_PREC_F64 || P->bn < 64) return FTN_OK;
  double flops = 0;
  for (const GemmProb& g : P->probs) flops += 2.0 * g.M * g.N * g.K;
  if (flops < (double)(1 << 30)) return FTN_OK;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return FTN_OK;
  std::vector<std::shared_ptr<TdPlan>> cands{P};
  for (int cap_bn = P->bn / 2; cap_bn >= 32 && cap_bn >= P->bn / 4; cap_bn /= 2) {
    std::shared_ptr<TdPlan> Q;
    FTN_TRY(build_plan(ctx, A, B, n, ax, ay, fa, fb, out_perm, prec, Q, cap_bn));
    if (Q->bn != cands.back()->bn) cands.push_back(Q);
  }
  if (cands.size() < 2) return FTN_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FTN_CUDA(cudaEventCreate(&e0));
  FTN_CUDA(cudaEventCreate(&e1));
  ftn_status st = FTN_OK;
  size_t best = 0;
  float best_ms = 0;
  // each candidate: one run to warm up, then the best of three timed runs
  // (one sample alone let run-to-run noise of a few microseconds decide)
  for (size_t c = 0; c < cands.size() && st == FTN_OK; ++c) {
    st = run_plan(ctx, *cands[c], A, B, out, prec);
    float cand_ms = -1.0f;
    for (int rep = 0; rep < 3 && st == FTN_OK; ++rep) {
      cudaEventRecord(e0, ctx->stream);
      st = run_plan(ctx, *cands[c], A, B, out, prec);
      cudaEventRecord(e1, ctx->stream);
      float ms = 0;
      if (st == FTN_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
          (cand_ms < 0 || ms < cand_ms))
        cand_ms = ms;
    }
    if (st == FTN_OK && cand_ms >= 0 && (c == 0 || cand_ms < best_ms)) {
      best = c;
      best_ms = cand_ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != FTN_OK) return st;
  P = cands[best];
  plan_cache(ctx)[plan_key(A, B, n, ax, ay, fa, fb, out_perm, prec)] = P;
  return FTN_OK;
}

// ---- transposition / dagger -------------------------------------------------------
struct TrPlan {
  std::vector<PermJob> jobs;
  int64_t tiles = 0;
  int staged = 0;
  std::shared_ptr<DevTables> dev;
  PermJob* d_jobs = nullptr;
};

static std::unordered_map<std::string, std::shared_ptr<TrPlan>>& tr_cache(ftn_ctx ctx) {
  static std::map<ftn_ctx, std::unordered_map<std::string, std::shared_ptr<TrPlan>>> caches;
  std::lock_guard<std::mutex> lock(g_cache_mu);
  return caches[ctx];
}

// out leg u = in leg perm[u]; `fermionic` selects the Eq. (transposition) sign
ftn_status permute_impl(ftn_ctx ctx, ftn_tensor t, const int* perm, bool fermionic, bool flip_duals, ftn_tensor* out) {
  if (!ctx || !t || !out || (t->rank > 0 && !perm)) return set_error(FTN_EINVAL, "null argument");
  const int r = t->rank;
  bool seen[MAXR] = {};
  for (int u = 0; u < r; ++u) {
    if (perm[u] < 0 || perm[u] >= r || seen[perm[u]]) return set_error(FTN_EINVAL, "bad permutation");
    seen[perm[u]] = true;
  }
  int32_t d0[MAXR], d1[MAXR];
  uint8_t du[MAXR];
  for (int u = 0; u < r; ++u) {
    d0[u] = t->d0[perm[u]];
    d1[u] = t->d1[perm[u]];
    du[u] = flip_duals ? (uint8_t)(1 - t->dual[perm[u]]) : t->dual[perm[u]];
  }
  ftn_tensor o = *out;
  bool created = false;
  if (o) {
    if (!same_meta(o, r, d0, d1, du, t->parity, t->dtype))
      return set_error(FTN_EINVAL, "preallocated output has the wrong metadata");
    if ((uintptr_t)o->data & 15)  // the permute stores 16-byte vectors
      return set_error(FTN_EINVAL, "preallocated output must be 16-byte aligned");
  } else {
    FTN_TRY(make_tensor(ctx, r, d0, d1, du, t->parity, t->dtype, &o));
    created = true;
  }
  CacheKey key;
  key.meta(t).put<uint8_t>(fermionic).put<uint8_t>(((uintptr_t)t->data & 15) == 0).ints(perm, r);
  auto& cache = tr_cache(ctx);
  std::shared_ptr<TrPlan> P;
  auto it = cache.find(key.s);
  if (it != cache.end()) {
    P = it->second;
  } else {
    P = std::make_shared<TrPlan>();
    for (int64_t b = 0; b < nblocks(r, t->parity); ++b) {
      uint32_t m = block_mask(r, t->parity, b);
      uint32_t mo = 0;
      for (int u = 0; u < r; ++u) mo |= ((m >> perm[u]) & 1u) << u;
      int64_t dims[MAXR], dstr[MAXR];
      for (int k = 0; k < r; ++k) dims[k] = leg_dim(t, k, m);
      int64_t s = 1;
      for (int u = r - 1; u >= 0; --u) {
        dstr[perm[u]] = s;
        s *= dims[perm[u]];
      }
      int sg = fermionic ? inversion_parity(r, perm, m) : 0;
      int64_t dst = r == 0 ? 0 : o->offsets[mo >> 1];
      if (r == 0) {
        dims[0] = 1;
        dstr[0] = 1;
      }
      add_perm_job(P->jobs, P->tiles, r == 0 ? 1 : r, dims, dstr, t->offsets[b], dst, sg ? -1 : 1);
    }
    P->staged = finalize_perm_jobs(P->jobs, dtype_size(t->dtype), &P->tiles, ((uintptr_t)t->data & 15) == 0);
    if (!jobs_in_bounds(P->jobs, t->numel, o->numel)) {
      if (created) ftn_tensor_free(o);
      return set_error(FTN_EINVAL, "internal error: transposition plan out of bounds");
    }
    P->dev = std::make_shared<DevTables>();
    P->dev->ctx = ctx;
    void* d = nullptr;
    ftn_status st = upload_table(ctx, P->jobs.data(), P->jobs.size() * sizeof(PermJob), &d);
    if (st != FTN_OK) {
      if (created) ftn_tensor_free(o);
      return st;
    }
    P->dev->p = d;
    P->d_jobs = (PermJob*)d;
    if (cache.size() > 65536) cache.clear();
    cache[key.s] = P;
  }
  int rec = prof_begin(ctx, "permute", 2.0 * t->numel * dtype_size(t->dtype), 0);
  ftn_status st = launch_permute(ctx, P->d_jobs, (int)P->jobs.size(), P->tiles, P->staged, t->data, o->data,
                                 nullptr, t->dtype, PERM_SAME);
  prof_end(ctx, rec);
  if (st != FTN_OK) {
    if (created) ftn_tensor_free(o);
    return st;
  }
  *out = o;
  return FTN_OK;
}

void clear_plan_caches(ftn_ctx ctx) {
  plan_cache(ctx).clear();
  tr_cache(ctx).clear();
  clear_grad_caches(ctx);
}

}  // namespace ftn

using namespace ftn;

extern "C" {

ftn_status ftn_tensordot(ftn_ctx ctx, ftn_tensor A, ftn_tensor B, int n, const int* axes_a, const int* axes_b,
                         uint64_t flip_a, uint64_t flip_b, const int* out_perm, ftn_prec prec, ftn_tensor* C) {
  return tensordot_impl(ctx, A, B, n, axes_a, axes_b, flip_a, flip_b, out_perm, prec, C);
}

ftn_status ftn_tensor_transpose(ftn_ctx ctx, ftn_tensor t, const int* perm, ftn_tensor* out) {
  return permute_impl(ctx, t, perm, true, false, out);
}

ftn_status ftn_tensor_dagger(ftn_ctx ctx, ftn_tensor t, ftn_tensor* out) {
  if (!t) return set_error(FTN_EINVAL, "null tensor");
  int perm[MAXR];
  for (int u = 0; u < t->rank; ++u) perm[u] = t->rank - 1 - u;
  return permute_impl(ctx, t, perm, false, true, out);
}

}  // extern "C"
