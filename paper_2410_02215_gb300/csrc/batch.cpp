// Batched execution of many independent contractions: job collectors that
// merge the kernel tables of many single-call plans into one launch per
// kernel, and the batched tensordot, normalisation and cast built on them.
#include "batch.h"

#include <algorithm>
#include <cstring>

namespace ftn {

ftn_status normalize_tensor(ftn_ctx ctx, ftn_tensor t, void* d_state, int step);
ftn_status cast_tensor(ftn_ctx ctx, ftn_tensor t, ftn_dtype to, ftn_tensor* out);
ftn_status tensordot_impl(ftn_ctx ctx, ftn_tensor A, ftn_tensor B, int n, const int* ax, const int* ay,
                          uint64_t flip_a, uint64_t flip_b, const int* out_perm, ftn_prec prec, ftn_tensor* C);

namespace {

// Small host tables packed at 256-byte offsets, uploaded with one copy.
struct TablePack {
  std::vector<uint8_t> host;
  size_t put(const void* p, size_t bytes) {
    const size_t off = (host.size() + 255) & ~(size_t)255;
    host.resize(off + bytes);
    if (bytes) std::memcpy(host.data() + off, p, bytes);
    return off;
  }
  ftn_status upload(ftn_ctx ctx, DevTables& dev) {
    dev.ctx = ctx;
    if (host.empty()) host.resize(256);
    return upload_table(ctx, host.data(), host.size(), &dev.p);
  }
};

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

inline const char* lowest256(const char* p) { return (const char*)((uintptr_t)p & ~(uintptr_t)255); }

size_t perm_out_size(ftn_dtype in_type, int mode) {
  switch (mode) {
    case PERM_TF32:
    case PERM_TF32X2: return 4;
    case PERM_BF16:
    case PERM_BF16X2:
    case PERM_F16X2: return 2;
    default: return dtype_size(in_type);
  }
}

}  // namespace

// ---- sign-permute ----------------------------------------------------------------
void PermBatch::add(const std::vector<PermJob>& jobs, int64_t total_tiles, int staged, const void* src, void* dst) {
  auto& v = items[staged ? 1 : 0];
  for (size_t i = 0; i < jobs.size(); ++i) {
    const int64_t end = i + 1 < jobs.size() ? jobs[i + 1].tile_begin : total_tiles;
    v.push_back({jobs[i], end - jobs[i].tile_begin, (const char*)src, (char*)dst});
  }
}

ftn_status flush_perm(ftn_ctx ctx, PermBatch& pb, ftn_dtype in_type, int mode, int64_t lo_delta) {
  const size_t es_in = dtype_size(in_type), es_out = perm_out_size(in_type, mode);
  for (int kind = 0; kind < 2; ++kind) {
    auto& v = pb.items[kind];
    if (v.empty()) continue;
    const char *sb = v[0].src, *db = v[0].dst;
    for (auto& it : v) {
      sb = std::min(sb, it.src);
      db = std::min(db, (const char*)it.dst);
    }
    sb = lowest256(sb);
    db = lowest256(db);
    const size_t bytes = v.size() * sizeof(PermJob);
    PermJob* jobs = (PermJob*)staging_begin(ctx, bytes);
    if (!jobs) return set_error(FTN_ENOMEM, "host staging allocation failed");
    int64_t tiles = 0;
    for (size_t i = 0; i < v.size(); ++i) {
      const auto& it = v[i];
      const int64_t ds = it.src - sb, dd = it.dst - db;
      if (ds % (int64_t)es_in || dd % (int64_t)es_out)
        return set_error(FTN_EINVAL, "batched permute: buffer not aligned to its element size");
      PermJob& j = jobs[i];
      j = it.j;
      j.src_off += ds / (int64_t)es_in;
      j.dst_off += dd / (int64_t)es_out;
      j.tile_begin = tiles;
      tiles += it.tiles;
    }
    DevTables dev;
    dev.ctx = ctx;
    FTN_TRY(staging_upload(ctx, bytes, &dev.p));
    char* d0 = const_cast<char*>(db);
    const int rec = prof_begin(ctx, "permute", 0, 0);
    const ftn_status st = launch_permute(ctx, (const PermJob*)dev.p, (int)v.size(), tiles, kind, sb, d0,
                                         lo_delta ? d0 + lo_delta : nullptr, in_type, mode);
    prof_end(ctx, rec);
    FTN_TRY(st);
  }
  pb.items[0].clear();
  pb.items[1].clear();
  return FTN_OK;
}

// ---- FP64 grouped GEMM -------------------------------------------------------------
void add_gemm_planned(GemmF64Batch& gb, const std::vector<GemmProb>& probs, int bn, const double* a, const double* b,
                      double* c) {
  auto& v = gb.by_bn[bn];
  for (const GemmProb& g : probs) v.push_back({g, a, b, c});
}

void add_reductions(GemmF64Batch& gb, const std::vector<GemmProb>& red, const double* part, double* c) {
  for (const GemmProb& r : red) gb.red.push_back({r, part, c});
}

ftn_status add_gemm_set(GemmF64Batch& gb, std::vector<GemmProb>& probs, const double* a, const double* b, double* c,
                        int64_t a_n, int64_t b_n, int64_t c_n) {
  if (probs.empty()) return FTN_OK;
  int max_n = 1;
  for (auto& g : probs) max_n = std::max(max_n, g.N);
  const int bn = f64_pick_bn(max_n);
  for (auto& g : probs) g.tiles_n = (g.N + bn - 1) / bn;
  int64_t tiles = 0;
  bool presplit = false;
  for (auto& g : probs) {
    g.tile_begin = tiles;
    tiles += (int64_t)g.tiles_m * g.tiles_n * (g.nsplit > 1 ? g.nsplit : 1);
    presplit = presplit || g.nsplit > 1;
  }
  std::vector<GemmProb> red;
  int64_t red_total = 0, part_n = 0;
  if (!presplit) part_n = plan_splitk_f64(probs, gb.ctx->num_sms, red, tiles, red_total);
  if (!probs_in_bounds(probs, a_n, b_n, part_n ? part_n : c_n) || (part_n && !red_in_bounds(red, part_n, c_n)))
    return set_error(FTN_EINVAL, "internal error: FP64 GEMM out of bounds");
  if (!part_n) {
    add_gemm_planned(gb, probs, bn, a, b, c);
    return FTN_OK;
  }
  double* part = (double*)dev_alloc(gb.ctx, (size_t)part_n * 8);
  if (!part) return set_error(FTN_ENOMEM, "device allocation failed (split-K partials)");
  gb.scratch.push_back(part);
  add_gemm_planned(gb, probs, bn, a, b, part);
  add_reductions(gb, red, part, c);
  return FTN_OK;
}

ftn_status flush_gemm_f64(GemmF64Batch& gb) {
  ftn_ctx ctx = gb.ctx;
  struct L {
    size_t off;
    int n, bn;  // bn 0: the warp kernel's launch (its items follow the problems at items_off)
    int64_t tiles;
    const char* base;
    std::vector<const GemmF64Batch::Item*> v;
  };
  // tiled problems by tile width, then every small problem in one warp launch
  std::vector<L> launches;
  L small{0, 0, 0, 0, nullptr, {}};
  for (auto& kv : gb.by_bn) {
    L l{0, 0, kv.first, 0, nullptr, {}};
    for (auto& it : kv.second) (f64w_small(it.g) ? small : l).v.push_back(&it);
    if (!l.v.empty()) launches.push_back(std::move(l));
  }
  if (!small.v.empty()) launches.push_back(std::move(small));
  size_t total = 0;
  for (L& l : launches) {
    const char* base = (const char*)l.v[0]->a;
    for (auto* it : l.v) base = std::min({base, (const char*)it->a, (const char*)it->b, (const char*)it->c});
    l.base = lowest256(base);
    l.n = (int)l.v.size();
    l.off = total;
    total = al256(total + l.v.size() * sizeof(GemmProb));
  }
  std::vector<WarpItem> witems;
  for (L& l : launches)
    if (l.bn == 0)
      for (int i = 0; i < l.n; ++i) f64w_items(l.v[i]->g, i, witems);
  const size_t items_off = total;
  total = al256(total + witems.size() * sizeof(WarpItem));
  const int nred = (int)gb.red.size();
  const size_t red_off = total;
  const char *pb = nullptr, *cb = nullptr;
  if (nred) {
    pb = (const char*)gb.red[0].part;
    cb = (const char*)gb.red[0].c;
    for (auto& it : gb.red) {
      pb = std::min(pb, (const char*)it.part);
      cb = std::min(cb, (const char*)it.c);
    }
    pb = lowest256(pb);
    cb = lowest256(cb);
    total += nred * sizeof(GemmProb);
  }
  if (launches.empty() && !nred) return FTN_OK;
  uint8_t* h = (uint8_t*)staging_begin(ctx, total);
  if (!h) return set_error(FTN_ENOMEM, "host staging allocation failed");
  double fl = 0;
  for (L& l : launches) {
    GemmProb* out = (GemmProb*)(h + l.off);
    int64_t tiles = 0;
    for (int i = 0; i < l.n; ++i) {
      const auto& it = *l.v[i];
      const int64_t da = (const char*)it.a - l.base, db = (const char*)it.b - l.base, dc = (const char*)it.c - l.base;
      if ((da | db | dc) & 7) return set_error(FTN_EINVAL, "batched GEMM: buffer not 8-byte aligned");
      GemmProb& g = out[i];
      g = it.g;
      g.a_off += da / 8;
      g.b_off += db / 8;
      g.c_off += dc / 8;
      g.tile_begin = tiles;
      if (l.bn) tiles += (int64_t)g.tiles_m * g.tiles_n * (g.nsplit > 1 ? g.nsplit : 1);
      fl += 2.0 * g.M * g.N * g.K;
    }
    l.tiles = tiles;
  }
  if (!witems.empty()) std::memcpy(h + items_off, witems.data(), witems.size() * sizeof(WarpItem));
  int64_t red_total = 0;
  if (nred) {
    GemmProb* out = (GemmProb*)(h + red_off);
    for (int i = 0; i < nred; ++i) {
      const auto& it = gb.red[i];
      const int64_t dp = (const char*)it.part - pb, dc = (const char*)it.c - cb;
      if ((dp | dc) & 7) return set_error(FTN_EINVAL, "batched reduction: buffer not 8-byte aligned");
      GemmProb& r = out[i];
      r = it.r;
      r.a_off += dp / 8;
      r.c_off += dc / 8;
      r.tile_begin = red_total;
      red_total += (int64_t)r.M * r.N;
    }
  }
  DevTables dev;
  dev.ctx = ctx;
  FTN_TRY(staging_upload(ctx, total, &dev.p));
  const uint8_t* d = (const uint8_t*)dev.p;
  const int rec = prof_begin(ctx, "gemm_f64", 0, fl);
  ftn_status st = FTN_OK;
  for (const L& l : launches) {
    const double* base = (const double*)l.base;
    if (l.bn)
      st = launch_gemm_f64(ctx, (const GemmProb*)(d + l.off), l.n, l.tiles, base, base, const_cast<double*>(base),
                           l.bn);
    else
      st = launch_gemm_f64_warp(ctx, (const GemmProb*)(d + l.off), (const WarpItem*)(d + items_off),
                                (int)witems.size(), base, base, const_cast<double*>(base));
    if (st != FTN_OK) break;
  }
  if (st == FTN_OK && nred)
    st = launch_splitk_reduce(ctx, (const GemmProb*)(d + red_off), nred, red_total, (const double*)pb,
                              (double*)const_cast<char*>(cb));
  prof_end(ctx, rec);
  gb.by_bn.clear();
  gb.red.clear();
  return st;
}

// ---- tensordot -------------------------------------------------------------------
ftn_status tensordot_batch(ftn_ctx ctx, std::vector<TdItem>& items, ftn_prec prec) {
  if (items.empty()) return FTN_OK;
  if (items.size() == 1) {
    TdItem& it = items[0];
    it.C = nullptr;
    return tensordot_impl(ctx, it.A, it.B, it.n, it.ax, it.ay, it.fa, it.fb, nullptr, prec, &it.C);
  }
  if (!prec_valid(prec)) return set_error(FTN_EINVAL, "bad precision");
  const bool tc = prec != FTN_PREC_F64;
  const bool split = prec_split(prec);
  const bool bf16 = prec_half(prec);  // 16-bit operands
  const ftn_dtype dt = tc ? FTN_F32 : FTN_F64;
  const size_t es = tc ? (bf16 ? 2 : 4) : 8, in_es = dtype_size(dt);
  std::vector<std::shared_ptr<TdPlan>> plans(items.size());
  struct Guard {
    std::vector<TdItem>& v;
    bool ok = false;
    ~Guard() {
      if (ok) return;
      for (auto& it : v) {
        ftn_tensor_free(it.C);
        it.C = nullptr;
      }
    }
  } guard{items};
  for (auto& it : items) it.C = nullptr;
  for (size_t i = 0; i < items.size(); ++i) {
    TdItem& it = items[i];
    if (!it.A || !it.B) return set_error(FTN_EINVAL, "null argument");
    if (it.A->dtype != dt || it.B->dtype != dt)
      return set_error(FTN_EUNSUPPORTED, "tensor dtype does not match the precision");
    FTN_TRY(validate_pairs(it.A, it.B, it.n, it.ax, it.ay));
    FTN_TRY(get_plan(ctx, it.A, it.B, it.n, it.ax, it.ay, it.fa, it.fb, nullptr, prec, plans[i]));
    const TdPlan& P = *plans[i];
    FTN_TRY(make_tensor(ctx, P.cr, P.cd0, P.cd1, P.cdual, P.cpar, dt, &it.C));
  }
  // workspace: [hi planes | lo planes (same layout) | plain results | FP64 split-K partials]
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  std::vector<size_t> o_a(items.size()), o_b(items.size()), o_c(items.size()), o_p(items.size());
  size_t hi = 0;
  for (size_t i = 0; i < items.size(); ++i) {
    o_a[i] = hi;
    hi += al((size_t)plans[i]->af_elems * es);
    o_b[i] = hi;
    hi += al((size_t)plans[i]->bf_elems * es);
  }
  size_t off = hi * (split ? 2 : 1);
  for (size_t i = 0; i < items.size(); ++i) {
    o_c[i] = off;
    off += plans[i]->fused ? 0 : al((size_t)plans[i]->tmp_numel * in_es);
  }
  for (size_t i = 0; i < items.size(); ++i) {
    o_p[i] = off;
    off += al((size_t)plans[i]->part_elems * 8);
  }
  uint8_t* ws = (uint8_t*)workspace(ctx, off);
  if (!ws) return set_error(FTN_ENOMEM, "workspace allocation failed");
  const int mode = prec_perm_mode(prec);
  // ---- 1. operands into fused sector matrices ----
  PermBatch pb;
  for (size_t i = 0; i < items.size(); ++i) {
    const TdPlan& P = *plans[i];
    pb.add(P.ja, P.ta, P.sa, items[i].A->data, ws + o_a[i]);
    pb.add(P.jb, P.tb, P.sb, items[i].B->data, ws + o_b[i]);
  }
  FTN_TRY(flush_perm(ctx, pb, dt, mode, split ? (int64_t)hi : 0));
  // ---- 2. grouped sector GEMMs ----
  auto target = [&](size_t i) -> void* { return plans[i]->fused ? items[i].C->data : (void*)(ws + o_c[i]); };
  if (!tc) {
    GemmF64Batch gb(ctx);
    for (size_t i = 0; i < items.size(); ++i) {
      const TdPlan& P = *plans[i];
      const double* a = (const double*)(ws + o_a[i]);
      const double* b = (const double*)(ws + o_b[i]);
      if (P.part_elems) {
        double* part = (double*)(ws + o_p[i]);
        add_gemm_planned(gb, P.probs, P.bn, a, b, part);
        add_reductions(gb, P.red, part, (double*)target(i));
      } else {
        add_gemm_planned(gb, P.probs, P.bn, a, b, (double*)target(i));
      }
    }
    FTN_TRY(flush_gemm_f64(gb));
  } else {
    std::map<int, std::vector<size_t>> by_bn;
    for (size_t i = 0; i < items.size(); ++i)
      if (plans[i]->n_tiled > 0) by_bn[plans[i]->bn].push_back(i);
    for (auto& kv : by_bn) {
      const int bn = kv.first;
      const auto& idx = kv.second;
      const char* cb = (const char*)target(idx[0]);
      for (size_t i : idx) cb = std::min(cb, (const char*)target(i));
      cb = lowest256(cb);
      size_t np = 0;
      for (size_t i : idx) np += plans[i]->n_tiled;
      const size_t om = 0, op = al256(2 * idx.size() * sizeof(TcMapSet));
      uint8_t* h = (uint8_t*)staging_begin(ctx, op + np * sizeof(GemmProb));
      if (!h) return set_error(FTN_ENOMEM, "host staging allocation failed");
      TcMapSet* maps = (TcMapSet*)(h + om);
      GemmProb* probs = (GemmProb*)(h + op);
      size_t p0 = 0;
      int64_t tiles = 0;
      double fl = 0;
      for (size_t q = 0; q < idx.size(); ++q) {
        const size_t i = idx[q];
        const TdPlan& P = *plans[i];
        TcOperands ops;
        for (int pi = 0; pi < 2; ++pi) {
          ops.a_hi[pi] = ws + o_a[i] + P.afoff[pi] * es;
          ops.b_hi[pi] = ws + o_b[i] + P.bfoff[pi] * es;
          ops.a_lo[pi] = split ? ws + hi + o_a[i] + P.afoff[pi] * es : nullptr;
          ops.b_lo[pi] = split ? ws + hi + o_b[i] + P.bfoff[pi] * es : nullptr;
          ops.a_rows[pi] = P.M[pi];
          ops.b_rows[pi] = P.N[pi];
          ops.kdim[pi] = (int32_t)P.K[pi];
          ops.ldk[pi] = (int32_t)P.ldk[pi];
        }
        for (int pi = 0; pi < 2; ++pi) FTN_TRY(tc_encode_set(prec, bn, ops, pi, &maps[2 * q + pi]));
        const int64_t dc = (const char*)target(i) - cb;
        if (dc & 3) return set_error(FTN_EINVAL, "batched GEMM: output not 4-byte aligned");
        for (int j = 0; j < P.n_tiled; ++j) {
          const GemmProb& g0 = P.probs[j];
          GemmProb& g = probs[p0 + j];
          g = g0;
          g.pi = (int32_t)(2 * q) + g0.pi;
          g.tile_begin += tiles;
          g.grp_first += (int32_t)p0;
          g.c_off += dc / 4;
          fl += 2.0 * g.M * g.N * g.K;
        }
        p0 += P.n_tiled;
        tiles += P.gemm_tiles;
      }
      DevTables dev;
      dev.ctx = ctx;
      FTN_TRY(staging_upload(ctx, op + np * sizeof(GemmProb), &dev.p));
      const uint8_t* d = (const uint8_t*)dev.p;
      const int rec = prof_begin(ctx, "gemm_tc", 0, fl);
      const ftn_status st = launch_gemm_tc_maps(ctx, prec, (const TcMapSet*)(d + om), (const GemmProb*)(d + op),
                                                (int)np, tiles, bn, (float*)const_cast<char*>(cb));
      prof_end(ctx, rec);
      FTN_TRY(st);
    }
    // the small problems of every plan in one CUDA-core launch: operands
    // rebased onto the workspace (lo planes `hi` bytes after the hi ones),
    // outputs onto the lowest target
    std::vector<GemmProb> sp;
    std::vector<WarpItem> wi;
    const char* cb = nullptr;
    for (size_t i = 0; i < items.size(); ++i)
      if ((size_t)plans[i]->n_tiled < plans[i]->probs.size())
        cb = cb ? std::min(cb, (const char*)target(i)) : (const char*)target(i);
    if (cb) {
      cb = lowest256(cb);
      double fl = 0;
      for (size_t i = 0; i < items.size(); ++i) {
        const TdPlan& P = *plans[i];
        const int64_t dc = (const char*)target(i) - cb;
        if (dc & 3) return set_error(FTN_EINVAL, "batched GEMM: output not 4-byte aligned");
        for (size_t j = (size_t)P.n_tiled; j < P.probs.size(); ++j) {
          GemmProb g = P.probs[j];
          g.a_off += (int64_t)(o_a[i] / es);
          g.b_off += (int64_t)(o_b[i] / es);
          g.c_off += dc / 4;
          fl += 2.0 * g.M * g.N * g.K;
          f64w_items(g, (int)sp.size(), wi);
          sp.push_back(g);
        }
      }
      TablePack tp;
      const size_t op = tp.put(sp.data(), sp.size() * sizeof(GemmProb));
      const size_t oi = tp.put(wi.data(), wi.size() * sizeof(WarpItem));
      DevTables dev;
      FTN_TRY(tp.upload(ctx, dev));
      const uint8_t* d = (const uint8_t*)dev.p;
      const int rec = prof_begin(ctx, "gemm_tc", 0, fl);
      const ftn_status st = launch_gemm_f32_warp(ctx, prec, (const GemmProb*)(d + op), (const WarpItem*)(d + oi),
                                                 (int)wi.size(), ws, ws, split ? (int64_t)(hi / es) : 0,
                                                 (float*)const_cast<char*>(cb));
      prof_end(ctx, rec);
      FTN_TRY(st);
    }
  }
  // ---- 3. plain results into the final layout ----
  PermBatch pc;
  for (size_t i = 0; i < items.size(); ++i)
    if (!plans[i]->fused) pc.add(plans[i]->jc, plans[i]->tc, plans[i]->sc, ws + o_c[i], items[i].C->data);
  if (!pc.empty()) FTN_TRY(flush_perm(ctx, pc, dt, PERM_SAME, 0));
  guard.ok = true;
  return FTN_OK;
}

// ---- normalisation and casts --------------------------------------------------------
ftn_status normalize_batch(ftn_ctx ctx, const std::vector<NormItem>& items) {
  if (items.size() == 1) return normalize_tensor(ctx, items[0].t, items[0].d_state, items[0].step);
  for (ftn_dtype dt : {FTN_F64, FTN_F32}) {
    std::vector<NormJob> small, large;
    int64_t tiles = 0;
    for (const NormItem& it : items) {
      if (it.t->dtype != dt || it.t->numel == 0) continue;
      NormJob j;
      std::memset(&j, 0, sizeof(j));
      j.x = it.t->data;
      j.n = it.t->numel;
      j.logacc = (double*)it.d_state;
      j.words = (unsigned long long*)((char*)it.d_state + 8);
      j.cur = it.step & 1;
      if (j.n <= 65536) {
        small.push_back(j);
      } else {
        j.tile_begin = tiles;
        tiles += (j.n + NORM_TILE - 1) / NORM_TILE;
        large.push_back(j);
      }
    }
    if (small.empty() && large.empty()) continue;
    TablePack tp;
    const size_t os = tp.put(small.data(), small.size() * sizeof(NormJob));
    const size_t ol = tp.put(large.data(), large.size() * sizeof(NormJob));
    DevTables dev;
    FTN_TRY(tp.upload(ctx, dev));
    const uint8_t* d = (const uint8_t*)dev.p;
    FTN_TRY(launch_normalize_batch(ctx, dt, (const NormJob*)(d + os), (int)small.size(), (const NormJob*)(d + ol),
                                   (int)large.size(), tiles));
  }
  return FTN_OK;
}

ftn_status cast_batch(ftn_ctx ctx, const std::vector<ftn_tensor>& t, ftn_dtype to, std::vector<ftn_tensor>& out) {
  out.assign(t.size(), nullptr);
  if (t.size() == 1) return cast_tensor(ctx, t[0], to, &out[0]);
  struct Guard {
    std::vector<ftn_tensor>& v;
    bool ok = false;
    ~Guard() {
      if (ok) return;
      for (auto& x : v) {
        ftn_tensor_free(x);
        x = nullptr;
      }
    }
  } guard{out};
  for (size_t i = 0; i < t.size(); ++i)
    FTN_TRY(make_tensor(ctx, t[i]->rank, t[i]->d0, t[i]->d1, t[i]->dual, t[i]->parity, to, &out[i]));
  for (ftn_dtype from : {FTN_F64, FTN_F32}) {
    std::vector<CastJob> jobs;
    int64_t tiles = 0;
    for (size_t i = 0; i < t.size(); ++i) {
      if (t[i]->dtype != from || t[i]->numel == 0) continue;
      jobs.push_back({t[i]->data, out[i]->data, t[i]->numel, tiles});
      tiles += (t[i]->numel + CAST_TILE - 1) / CAST_TILE;
    }
    if (jobs.empty()) continue;
    TablePack tp;
    tp.put(jobs.data(), jobs.size() * sizeof(CastJob));
    DevTables dev;
    FTN_TRY(tp.upload(ctx, dev));
    FTN_TRY(launch_cast_batch(ctx, from, to, (const CastJob*)dev.p, (int)jobs.size(), tiles));
  }
  guard.ok = true;
  return FTN_OK;
}

}  // namespace ftn
