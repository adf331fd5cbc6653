// Adjoint of the fermionic tensordot (the contraction of Eq. standardcontract
// with the arrow rule of Eq. fermionictn2 is linear in each operand).
//
// The forward contraction multiplies every block pair by one sign that is a
// function of parity bits only:  C_blk = s_out s_A s_B (A_blk . B_blk) in the
// fused sector-matrix coordinates (s_A: transposition of A into [free | bond]
// with the bond's arrow parity and the extra bond parities, s_B: the same for
// B, s_out: the output transposition).  For L = sum(G * C) therefore
//     dA_fused = (s_out G)_fused . (s_B B)_fused^T   then   dA = s_A * dA_fused,
// summed over every column block of the sector; dB likewise with the roles of
// A and B exchanged.  On the GPU: one sign-permute of G into the fused result
// layout, one of the other operand into a [bond | free] layout, and one
// grouped sector GEMM whose epilogue writes straight into the differentiated
// operand's block layout with its sign.
#include <algorithm>
#include <map>
#include <mutex>

#include "tdplan.h"

namespace ftn {

namespace {

struct GradPlan {
  bool wrt_b = false;
  // per bond-parity sector pi: rows of the result (free combos of the
  // differentiated operand), contraction length (free combos of the other
  // operand), bond combos; leading dimension of both GEMM operands
  int64_t R[2] = {0, 0}, L[2] = {0, 0}, K[2] = {0, 0}, ld[2] = {8, 8};
  int64_t goff[2] = {0, 0}, yoff[2] = {0, 0};
  int64_t g_elems = 0, y_elems = 0;
  std::vector<PermJob> jg, jy;
  int64_t tg = 0, ty = 0;
  int sg = 0, sy = 0;
  std::vector<GemmProb> probs, red;
  int64_t tiles = 0, part_elems = 0, red_total = 0;
  bool tc_parts = false;  // tensor-core path: every problem writes FP32 partial slabs, reduced in FP64
  int bn = 0;
  int32_t xd0[MAXR], xd1[MAXR];
  uint8_t xdu[MAXR];
  int xrank = 0, xpar = 0;
  int cr = 0, cpar = 0;
  int32_t cd0[MAXR], cd1[MAXR];
  uint8_t cdu[MAXR];
  std::shared_ptr<DevTables> dev;
  PermJob* d_jg = nullptr;
  PermJob* d_jy = nullptr;
  GemmProb* d_probs = nullptr;
  GemmProb* d_red = nullptr;
};

std::mutex g_grad_mu;

std::unordered_map<std::string, std::shared_ptr<GradPlan>>& grad_cache(ftn_ctx ctx) {
  static std::map<ftn_ctx, std::unordered_map<std::string, std::shared_ptr<GradPlan>>> caches;
  std::lock_guard<std::mutex> lock(g_grad_mu);
  return caches[ctx];
}

ftn_status upload(ftn_ctx ctx, GradPlan& P) {
  const size_t a = P.jg.size() * sizeof(PermJob), b = P.jy.size() * sizeof(PermJob),
               c = P.probs.size() * sizeof(GemmProb), d = P.red.size() * sizeof(GemmProb);
  std::vector<uint8_t> host(a + b + c + d + 16);
  std::memcpy(host.data(), P.jg.data(), a);
  std::memcpy(host.data() + a, P.jy.data(), b);
  std::memcpy(host.data() + a + b, P.probs.data(), c);
  if (d) std::memcpy(host.data() + a + b + c, P.red.data(), d);
  P.dev = std::make_shared<DevTables>();
  P.dev->ctx = ctx;
  void* dp = nullptr;
  FTN_TRY(upload_table(ctx, host.data(), a + b + c + d, &dp));
  P.dev->p = dp;
  uint8_t* base = (uint8_t*)dp;
  P.d_jg = (PermJob*)base;
  P.d_jy = (PermJob*)(base + a);
  P.d_probs = (GemmProb*)(base + a + b);
  P.d_red = d ? (GemmProb*)(base + a + b + c) : nullptr;
  return FTN_OK;
}

// Row-major strides of a block of t (mask m), leg by leg.
void block_strides(const ftn_tensor_s* t, uint32_t m, int64_t* dims, int64_t* str) {
  int64_t s = 1;
  for (int k = t->rank - 1; k >= 0; --k) {
    dims[k] = leg_dim(t, k, m);
    str[k] = s;
    s *= dims[k];
  }
}

ftn_status build(ftn_ctx ctx, const ftn_tensor_s* A, const ftn_tensor_s* B, const ftn_tensor_s* G, int n,
                 const int* ax, const int* ay, uint64_t flip_a, uint64_t flip_b, const int* out_perm, ftn_prec prec,
                 bool wrt_b, std::shared_ptr<GradPlan>& out) {
  auto P = std::make_shared<GradPlan>();
  P->wrt_b = wrt_b;
  const bool tc = prec != FTN_PREC_F64;
  int fa[MAXR], fb[MAXR], nfa = 0, nfb = 0;
  bool in_a[MAXR] = {}, in_b[MAXR] = {};
  for (int i = 0; i < n; ++i) in_a[ax[i]] = in_b[ay[i]] = true;
  for (int k = 0; k < A->rank; ++k)
    if (!in_a[k]) fa[nfa++] = k;
  for (int k = 0; k < B->rank; ++k)
    if (!in_b[k]) fb[nfb++] = k;
  const int pA = A->parity, pB = B->parity;
  int64_t fad0[MAXR], fad1[MAXR], fbd0[MAXR], fbd1[MAXR], kd0[MAXR], kd1[MAXR];
  for (int j = 0; j < nfa; ++j) fad0[j] = A->d0[fa[j]], fad1[j] = A->d1[fa[j]];
  for (int j = 0; j < nfb; ++j) fbd0[j] = B->d0[fb[j]], fbd1[j] = B->d1[fb[j]];
  for (int i = 0; i < n; ++i) kd0[i] = A->d0[ax[i]], kd1[i] = A->d1[ax[i]];
  std::vector<int64_t> rowoff[2], rowsz[2], coloff[2], colsz[2], koff[2], ksz[2];
  int64_t M[2], N[2];
  for (int pi = 0; pi < 2; ++pi) {
    M[pi] = sector_offsets(nfa, fad0, fad1, pA ^ pi, rowoff[pi], rowsz[pi]);
    N[pi] = sector_offsets(nfb, fbd0, fbd1, pB ^ pi, coloff[pi], colsz[pi]);
    P->K[pi] = sector_offsets(n, kd0, kd1, pi, koff[pi], ksz[pi]);
    P->R[pi] = wrt_b ? N[pi] : M[pi];
    P->L[pi] = wrt_b ? M[pi] : N[pi];
    P->ld[pi] = std::max<int64_t>(8, (P->L[pi] + 7) / 8 * 8);
  }
  P->goff[1] = (P->R[0] * P->ld[0] + 63) / 64 * 64;
  P->g_elems = P->goff[1] + P->R[1] * P->ld[1];
  P->yoff[1] = (P->K[0] * P->ld[0] + 63) / 64 * 64;
  P->y_elems = P->yoff[1] + P->K[1] * P->ld[1];

  // ---- G (final result layout) -> fused: rows = differentiated operand's free combos ----
  const int cr = nfa + nfb;
  int perm[MAXR];
  for (int u = 0; u < cr; ++u) perm[u] = out_perm ? out_perm[u] : u;
  P->cr = cr;
  P->cpar = pA ^ pB;
  for (int u = 0; u < cr; ++u) {
    const int t = perm[u];
    const ftn_tensor_s* src = t < nfa ? A : B;
    const int leg = t < nfa ? fa[t] : fb[t - nfa];
    P->cd0[u] = src->d0[leg];
    P->cd1[u] = src->d1[leg];
    P->cdu[u] = src->dual[leg];
  }
  if (G->rank != cr || G->parity != P->cpar) return set_error(FTN_ESHAPE, "gradient of the result has the wrong rank or parity");
  for (int u = 0; u < cr; ++u)
    if (G->d0[u] != P->cd0[u] || G->d1[u] != P->cd1[u] || G->dual[u] != P->cdu[u])
      return set_error(FTN_ESHAPE, "gradient of the result has the wrong legs");
  for (int64_t b = 0; b < nblocks(cr, G->parity); ++b) {
    const uint32_t mo = block_mask(cr, G->parity, b);
    uint32_t m = 0;  // the same block in the unpermuted order [A free | B free]
    for (int u = 0; u < cr; ++u) m |= ((mo >> u) & 1u) << perm[u];
    const uint32_t mA = m & ((1u << nfa) - 1u), mB = m >> nfa;
    const int pi = (popc(mA) & 1) ^ pA;
    int64_t tdim[MAXR];  // dims of the unpermuted legs
    for (int u = 0; u < cr; ++u) tdim[perm[u]] = leg_dim(G, u, mo);
    int64_t tstr[MAXR];
    int64_t s = 1;
    if (!wrt_b) {  // rows A free (row stride ld), columns B free
      for (int j = nfb - 1; j >= 0; --j) tstr[nfa + j] = s, s *= tdim[nfa + j];
      s = P->ld[pi];
      for (int j = nfa - 1; j >= 0; --j) tstr[j] = s, s *= tdim[j];
    } else {  // rows B free, columns A free
      for (int j = nfa - 1; j >= 0; --j) tstr[j] = s, s *= tdim[j];
      s = P->ld[pi];
      for (int j = nfb - 1; j >= 0; --j) tstr[nfa + j] = s, s *= tdim[nfa + j];
    }
    int64_t dims[MAXR], dstr[MAXR];
    for (int u = 0; u < cr; ++u) dims[u] = tdim[perm[u]], dstr[u] = tstr[perm[u]];
    const int64_t dst = P->goff[pi] + (wrt_b ? coloff[pi][mB] * P->ld[pi] + rowoff[pi][mA]
                                             : rowoff[pi][mA] * P->ld[pi] + coloff[pi][mB]);
    const int sg = out_perm ? inversion_parity(cr, perm, m) : 0;
    add_perm_job(P->jg, P->tg, cr, dims, dstr, G->offsets[b], dst, sg ? -1 : 1);
  }
  // ---- the other operand -> [bond | free]: rows = bond combos, columns = its free combos ----
  int permA[MAXR], permB[MAXR];
  for (int j = 0; j < nfa; ++j) permA[j] = fa[j];
  for (int i = 0; i < n; ++i) permA[nfa + i] = ax[i];
  for (int i = 0; i < n; ++i) permB[i] = ay[n - 1 - i];
  for (int j = 0; j < nfb; ++j) permB[n + j] = fb[j];
  uint32_t arrow_a = 0;
  for (int i = 0; i < n; ++i)
    if (A->dual[ax[i]] == 0) arrow_a |= 1u << ax[i];
  auto sign_a = [&](uint32_t m) {
    return inversion_parity(A->rank, permA, m) ^ (popc(m & arrow_a) & 1) ^ (popc(m & (uint32_t)flip_a) & 1);
  };
  auto sign_b = [&](uint32_t m) { return inversion_parity(B->rank, permB, m) ^ (popc(m & (uint32_t)flip_b) & 1); };
  const ftn_tensor_s* Y = wrt_b ? A : B;
  const int* yf = wrt_b ? fa : fb;
  const int nyf = wrt_b ? nfa : nfb;
  const int* yk = wrt_b ? ax : ay;
  for (int64_t b = 0; b < nblocks(Y->rank, Y->parity); ++b) {
    const uint32_t m = block_mask(Y->rank, Y->parity, b);
    const uint32_t mF = gather_bits(m, yf, nyf), mK = gather_bits(m, yk, n);
    const int pi = popc(mK) & 1;
    int64_t dims[MAXR], dstr[MAXR];
    for (int k = 0; k < Y->rank; ++k) dims[k] = leg_dim(Y, k, m);
    int64_t s = 1;
    for (int j = nyf - 1; j >= 0; --j) dstr[yf[j]] = s, s *= dims[yf[j]];
    s = P->ld[pi];
    for (int i = n - 1; i >= 0; --i) dstr[yk[i]] = s, s *= dims[yk[i]];
    const int64_t dst = P->yoff[pi] + koff[pi][mK] * P->ld[pi] + (wrt_b ? rowoff[pi][mF] : coloff[pi][mF]);
    const int sg = wrt_b ? sign_a(m) : sign_b(m);
    add_perm_job(P->jy, P->ty, Y->rank, dims, dstr, Y->offsets[b], dst, sg ? -1 : 1);
  }
  P->sg = finalize_perm_jobs(P->jg, dtype_size(G->dtype), &P->tg, ((uintptr_t)G->data & 15) == 0);
  P->sy = finalize_perm_jobs(P->jy, dtype_size(Y->dtype), &P->ty, ((uintptr_t)Y->data & 15) == 0);

  // ---- GEMM problems: one per block of the differentiated operand ----
  const ftn_tensor_s* X = wrt_b ? B : A;
  const int* xf = wrt_b ? fb : fa;
  const int nxf = wrt_b ? nfb : nfa;
  const int* xk = wrt_b ? ay : ax;
  P->xrank = X->rank;
  P->xpar = X->parity;
  for (int k = 0; k < X->rank; ++k) P->xd0[k] = X->d0[k], P->xd1[k] = X->d1[k], P->xdu[k] = X->dual[k];
  int maxN = 1;
  for (int64_t b = 0; b < nblocks(X->rank, X->parity); ++b) {
    const uint32_t m = block_mask(X->rank, X->parity, b);
    const uint32_t mF = gather_bits(m, xf, nxf), mK = gather_bits(m, xk, n);
    const int pi = popc(mK) & 1;
    const int64_t rows = wrt_b ? colsz[pi][mF] : rowsz[pi][mF];
    const int64_t cols = ksz[pi][mK];
    if (rows == 0 || cols == 0) continue;
    GemmProb g;
    std::memset(&g, 0, sizeof(g));
    g.M = (int32_t)rows;
    g.N = (int32_t)cols;
    g.K = (int32_t)P->L[pi];
    g.pi = pi;
    g.lda = g.ldb = (int32_t)P->ld[pi];
    g.a_row0 = (int32_t)(wrt_b ? coloff[pi][mF] : rowoff[pi][mF]);
    g.b_row0 = (int32_t)koff[pi][mK];
    g.a_off = P->goff[pi] + (int64_t)g.a_row0 * P->ld[pi];
    g.b_off = P->yoff[pi] + (int64_t)g.b_row0 * P->ld[pi];
    g.a_sm = g.b_sn = P->ld[pi];
    g.a_sk = g.b_sk = 1;
    int64_t dims[MAXR], str[MAXR];
    block_strides(X, m, dims, str);
    g.c_off = X->offsets[b];
    g.c_sign = (wrt_b ? sign_b(m) : sign_a(m)) ? -1 : 1;
    g.nrl = nxf;
    g.ncl = n;
    for (int j = 0; j < nxf; ++j) g.rdim[j] = (int32_t)dims[xf[j]], g.rstr[j] = str[xf[j]];
    for (int i = 0; i < n; ++i) g.cdim[i] = (int32_t)dims[xk[i]], g.cstr[i] = str[xk[i]];
    // stores run along the rows when the operand's last (contiguous) leg is a free one
    g.epi_rows = std::find(xf, xf + nxf, X->rank - 1) != xf + nxf ? 1 : 0;
    g.vec4 = 0;
    maxN = std::max(maxN, g.N);
    P->probs.push_back(g);
  }
  P->bn = tc ? tc_pick_bn(maxN, prec) : f64_pick_bn(maxN);
  for (GemmProb& g : P->probs) {
    g.tiles_m = tc ? (g.M + 127) / 128 : (g.M + 63) / 64;
    g.tiles_n = (g.N + P->bn - 1) / P->bn;
  }
  if (tc) {
    // Long contractions (the gradient of a small operand contracts over all
    // free states of the large one): K parts of at most TC_KPART elements,
    // and enough parts to give two tiles per SM.  The tensor core
    // accumulates each part in FP32; the parts are added in FP64.  If any
    // problem is split, every problem writes partial slabs (the kernel has
    // one output base) and one reduction writes the gradient.
    constexpr int TC_KPART = 2048, KALIGN = 64;  // a multiple of both TMA K boxes (32 TF32, 64 BF16)
    int64_t tiles0 = 0;
    for (const GemmProb& g : P->probs) tiles0 += (int64_t)g.tiles_m * g.tiles_n;
    const int64_t want = tiles0 > 0 ? (2 * (int64_t)ctx->num_sms + tiles0 - 1) / tiles0 : 1;
    bool need = false;
    for (const GemmProb& g : P->probs) need = need || g.K > TC_KPART || (want > 1 && g.K >= 8 * KALIGN);
    if (need) {
      std::vector<GemmProb> parts;
      int64_t part = 0, elems = 0;
      for (const GemmProb& g : P->probs) {
        int s = (int)std::max<int64_t>((g.K + TC_KPART - 1) / TC_KPART, std::min<int64_t>(want, g.K / (4 * KALIGN)));
        s = std::max(1, std::min(s, 256));
        int kchunk = (g.K + s - 1) / s;
        kchunk = std::max(KALIGN, (kchunk + KALIGN - 1) / KALIGN * KALIGN);
        s = std::max(1, (g.K + kchunk - 1) / kchunk);
        const int64_t mn = (int64_t)g.M * g.N;
        GemmProb r = g;  // reduction job: the original epilogue
        r.a_off = part;
        r.nsplit = s;
        r.c_slab = mn;
        r.tile_begin = elems;
        P->red.push_back(r);
        for (int q = 0; q < s; ++q) {
          GemmProb h = g;
          h.k0 = q * kchunk;
          h.K = std::min(kchunk, g.K - h.k0);
          gemm_plain_output(h, part + (int64_t)q * mn, g.N);
          h.epi_rows = 0;
          h.vec4 = (g.N % 4 == 0 && (part + (int64_t)q * mn) % 4 == 0) ? 1 : 0;
          parts.push_back(h);
        }
        part += mn * s;
        elems += mn;
      }
      P->probs.swap(parts);
      P->part_elems = part;
      P->red_total = elems;
      P->tc_parts = true;
    }
    std::stable_sort(P->probs.begin(), P->probs.end(), [](const GemmProb& x, const GemmProb& y) {
      if (x.pi != y.pi) return x.pi < y.pi;
      if (x.a_row0 != y.a_row0) return x.a_row0 < y.a_row0;
      return x.b_row0 < y.b_row0;
    });
    for (size_t i = 0; i < P->probs.size();) {
      size_t j = i;
      int32_t row_tiles = 0;
      while (j < P->probs.size() && P->probs[j].pi == P->probs[i].pi && P->probs[j].a_row0 == P->probs[i].a_row0) {
        P->probs[j].tn_off = row_tiles;
        row_tiles += P->probs[j].tiles_n;
        ++j;
      }
      for (size_t q = i; q < j; ++q) {
        P->probs[q].grp_first = (int32_t)i;
        P->probs[q].grp_count = (int32_t)(j - i);
        P->probs[q].row_tiles = row_tiles;
        P->probs[q].tile_begin = P->tiles;
      }
      P->tiles += (int64_t)P->probs[i].tiles_m * row_tiles;
      i = j;
    }
  } else {
    for (GemmProb& g : P->probs) {
      g.tile_begin = P->tiles;
      P->tiles += (int64_t)g.tiles_m * g.tiles_n;
    }
    P->part_elems = plan_splitk_f64(P->probs, ctx->num_sms, P->red, P->tiles, P->red_total);
  }
  const int64_t x_numel = X->numel;
  bool k_ok = true;  // K parts stay inside the contraction and start on a TMA box boundary
  for (const GemmProb& g : P->probs) k_ok = k_ok && g.k0 >= 0 && g.k0 % 64 == 0 && g.k0 + g.K <= P->L[g.pi];
  if (!k_ok || !jobs_in_bounds(P->jg, G->numel, P->g_elems) || !jobs_in_bounds(P->jy, Y->numel, P->y_elems) ||
      !probs_in_bounds(P->probs, P->g_elems, P->y_elems, P->part_elems ? P->part_elems : x_numel) ||
      (P->part_elems && !red_in_bounds(P->red, P->part_elems, x_numel)))
    return set_error(FTN_EINVAL, "internal error: gradient plan out of bounds");
  FTN_TRY(upload(ctx, *P));
  out = P;
  return FTN_OK;
}

ftn_status get_grad_plan(ftn_ctx ctx, const ftn_tensor_s* A, const ftn_tensor_s* B, const ftn_tensor_s* G, int n,
                         const int* ax, const int* ay, uint64_t fa, uint64_t fb, const int* out_perm, ftn_prec prec,
                         bool wrt_b, std::shared_ptr<GradPlan>& P) {
  CacheKey key;
  key.put<uint8_t>(wrt_b).meta(A).meta(B).meta(G).ints(ax, n).ints(ay, n).put(fa).put(fb).put<int32_t>((int32_t)prec);
  key.put<uint8_t>(((uintptr_t)G->data & 15) == 0).put<uint8_t>(((uintptr_t)(wrt_b ? A : B)->data & 15) == 0);
  key.put<uint8_t>(out_perm != nullptr);
  if (out_perm) key.ints(out_perm, A->rank + B->rank - 2 * n);
  auto& cache = grad_cache(ctx);
  auto it = cache.find(key.s);
  if (it != cache.end()) {
    P = it->second;
    return FTN_OK;
  }
  FTN_TRY(build(ctx, A, B, G, n, ax, ay, fa, fb, out_perm, prec, wrt_b, P));
  if (cache.size() > 65536) cache.clear();
  cache[key.s] = P;
  return FTN_OK;
}

ftn_status run_grad(ftn_ctx ctx, const GradPlan& P, const ftn_tensor_s* G, const ftn_tensor_s* Y, ftn_prec prec,
                    ftn_tensor dX) {
  const bool tc = prec != FTN_PREC_F64;
  const bool split = prec_split(prec);
  const bool bf16 = prec_half(prec);  // 16-bit operands
  const size_t es = tc ? (bf16 ? 2 : 4) : 8;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t g_b = al((size_t)P.g_elems * es), y_b = al((size_t)P.y_elems * es);
  const size_t p_b = al((size_t)P.part_elems * (tc ? 4 : 8));
  const int planes = split ? 2 : 1;
  const size_t need = (g_b + y_b) * planes + p_b;
  uint8_t* ws = (uint8_t*)workspace(ctx, need);
  if (!ws) return set_error(FTN_ENOMEM, "workspace allocation failed");
  uint8_t* g_hi = ws;
  uint8_t* g_lo = split ? ws + g_b : nullptr;
  uint8_t* y_hi = ws + g_b * planes;
  uint8_t* y_lo = split ? y_hi + y_b : nullptr;
  const int mode = prec_perm_mode(prec);
  int rec = prof_begin(ctx, "permute", (double)G->numel * (dtype_size(G->dtype) + es * planes), 0);
  FTN_TRY(launch_permute(ctx, P.d_jg, (int)P.jg.size(), P.tg, P.sg, G->data, g_hi, g_lo, G->dtype, mode));
  FTN_TRY(launch_permute(ctx, P.d_jy, (int)P.jy.size(), P.ty, P.sy, Y->data, y_hi, y_lo, Y->dtype, mode));
  prof_end(ctx, rec);
  if (P.probs.empty()) return FTN_OK;
  double fl = 0;
  for (const GemmProb& g : P.probs) fl += 2.0 * g.M * g.N * g.K;
  if (!tc) {
    rec = prof_begin(ctx, "gemm_f64", 0, fl);
    if (P.part_elems) {
      double* part = (double*)(ws + need - p_b);
      FTN_TRY(launch_gemm_f64(ctx, P.d_probs, (int)P.probs.size(), P.tiles, (const double*)g_hi, (const double*)y_hi,
                              part, P.bn));
      FTN_TRY(launch_splitk_reduce(ctx, P.d_red, (int)P.red.size(), P.red_total, part, (double*)dX->data));
    } else {
      FTN_TRY(launch_gemm_f64(ctx, P.d_probs, (int)P.probs.size(), P.tiles, (const double*)g_hi, (const double*)y_hi,
                              (double*)dX->data, P.bn));
    }
    prof_end(ctx, rec);
    return FTN_OK;
  }
  TcOperands ops;
  for (int pi = 0; pi < 2; ++pi) {
    ops.a_hi[pi] = g_hi + P.goff[pi] * es;
    ops.b_hi[pi] = y_hi + P.yoff[pi] * es;
    ops.a_lo[pi] = split ? g_lo + P.goff[pi] * es : nullptr;
    ops.b_lo[pi] = split ? y_lo + P.yoff[pi] * es : nullptr;
    ops.a_rows[pi] = P.R[pi];
    ops.b_rows[pi] = P.K[pi];
    ops.kdim[pi] = (int32_t)P.L[pi];
    ops.ldk[pi] = (int32_t)P.ld[pi];
  }
  rec = prof_begin(ctx, "gemm_tc", 0, fl);
  if (P.tc_parts) {
    float* part = (float*)(ws + need - p_b);
    FTN_TRY(launch_gemm_tc(ctx, prec, ops, P.d_probs, (int)P.probs.size(), P.tiles, P.bn, part));
    FTN_TRY(launch_splitk_reduce_f32(ctx, P.d_red, (int)P.red.size(), P.red_total, part, (float*)dX->data));
  } else {
    FTN_TRY(launch_gemm_tc(ctx, prec, ops, P.d_probs, (int)P.probs.size(), P.tiles, P.bn, (float*)dX->data));
  }
  prof_end(ctx, rec);
  return FTN_OK;
}

}  // namespace

void clear_grad_caches(ftn_ctx ctx) { grad_cache(ctx).clear(); }

ftn_status tensordot_grad_impl(ftn_ctx ctx, ftn_tensor A, ftn_tensor B, ftn_tensor G, int n, const int* ax,
                               const int* ay, uint64_t flip_a, uint64_t flip_b, const int* out_perm, ftn_prec prec,
                               ftn_tensor* dA, ftn_tensor* dB) {
  if (!ctx || !A || !B || !G) return set_error(FTN_EINVAL, "null argument");
  if (A->dtype != B->dtype || G->dtype != A->dtype) return set_error(FTN_EINVAL, "A, B and G must have one dtype");
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
  for (int w = 0; w < 2; ++w) {
    ftn_tensor* pd = w ? dB : dA;
    if (!pd) continue;
    std::shared_ptr<GradPlan> P;
    FTN_TRY(get_grad_plan(ctx, A, B, G, n, ax, ay, flip_a, flip_b, out_perm, prec, w == 1, P));
    ftn_tensor out = *pd;
    bool created = false;
    if (out) {
      if (!same_meta(out, P->xrank, P->xd0, P->xd1, P->xdu, P->xpar, A->dtype))
        return set_error(FTN_EINVAL, "preallocated gradient has the wrong metadata");
      if ((uintptr_t)out->data & 15)  // the epilogues store 16-byte vectors
        return set_error(FTN_EINVAL, "preallocated gradient must be 16-byte aligned");
    } else {
      FTN_TRY(make_tensor(ctx, P->xrank, P->xd0, P->xd1, P->xdu, P->xpar, A->dtype, &out));
      created = true;
    }
    const ftn_status st = run_grad(ctx, *P, G, w ? A : B, prec, out);
    if (st != FTN_OK) {
      if (created) ftn_tensor_free(out);
      return st;
    }
    *pd = out;
  }
  return FTN_OK;
}

}  // namespace ftn

using namespace ftn;

extern "C" {

ftn_status ftn_tensordot_grad(ftn_ctx ctx, ftn_tensor A, ftn_tensor B, ftn_tensor G, int n, const int* axes_a,
                              const int* axes_b, uint64_t flip_a, uint64_t flip_b, const int* out_perm, ftn_prec prec,
                              ftn_tensor* dA, ftn_tensor* dB) {
  return tensordot_grad_impl(ctx, A, B, G, n, axes_a, axes_b, flip_a, flip_b, out_perm, prec, dA, dB);
}

}  // extern "C"
