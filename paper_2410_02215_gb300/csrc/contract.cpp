// Contraction-tree executor ftn_contract / ftn_contract_batch (Fig. 1;
// Secs. II.C-II.D; Sec. III) and the Hubbard operator tensors
// ftn_hubbard_term (Eq. fermi-hubbard-ham).
//
// The executor walks an SSA tree of pairwise contractions.  Locally ordered
// formalism (no positions): every step is op(a, b) with the bond parity of
// bonds contracted against their arrows.  Globally ordered formalism
// (positions given): the later tensor l of a step is moved left past every
// tensor c between the two positions -- each bond it shares with c carries
// the bond parity g (a flip on that leg of l) and each pair of odd tensors a
// phase (-1)^{p_l p_c} -- and the pair is then contracted as the plain
// ordered product F(e l) (arrow parities cancelled).  Compression (early or
// late, bonds above chi, neighbours in increasing id) uses ftn_compress; each
// new tensor is divided by its largest |entry| on the device with the natural
// log accumulated in FP64.
//
// Many networks run in lock step: round s performs step s of every network
// that has one -- the compressions before it (one sub-round per position in
// each network's own list, so a network's compressions keep their order),
// the pairwise contraction, the compressions after it and the normalisation
// -- each stage as one batched launch per kernel over all networks.  One
// network is the batch of one.
#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <set>

#include "batch.h"

namespace ftn {

ftn_status normalize_tensor(ftn_ctx ctx, ftn_tensor t, void* d_state, int step);
ftn_status cast_tensor(ftn_ctx ctx, ftn_tensor t, ftn_dtype to, ftn_tensor* out);

namespace {

struct Live {
  ftn_tensor t = nullptr;
  std::vector<int64_t> ids;  // leg identities
  int64_t pos = 0;
};

struct Exec {
  ftn_prec prec = FTN_PREC_F64;
  bool global = false;
  const ftn_tree* tree = nullptr;
  int n = 0;
  std::map<int64_t, Live> live;
  std::map<int64_t, int64_t> partner;  // leg id -> leg id
  std::map<int64_t, int64_t> owner;    // leg id -> tensor id
  std::map<int64_t, int> dummy;        // dummy leg id -> index of its odd tensor (locally ordered only)
  int64_t next_leg = 1ll << 40;
  int sign = 1;
  // when set, consumed tensors are handed here instead of freed (the
  // gradient executor keeps every operand of its tape)
  std::vector<ftn_tensor>* retain = nullptr;

  // The walk's state between two steps (the tensors are referred to, not
  // owned): taken at a checkpoint, put back to replay the steps after it.
  struct State {
    std::map<int64_t, Live> live;
    std::map<int64_t, int64_t> partner, owner;
    std::map<int64_t, int> dummy;
    int64_t next_leg = 0;
    int sign = 1;
  };
  void save(State& st) const {
    st.live = live;
    st.partner = partner;
    st.owner = owner;
    st.dummy = dummy;
    st.next_leg = next_leg;
    st.sign = sign;
  }
  void load(const State& st) {  // the current live tensors are the caller's to free
    live = st.live;
    partner = st.partner;
    owner = st.owner;
    dummy = st.dummy;
    next_leg = st.next_leg;
    sign = st.sign;
  }
  Exec() = default;
  Exec(const Exec&) = delete;
  Exec& operator=(const Exec&) = delete;
  ~Exec() {
    for (auto& kv : live) ftn_tensor_free(kv.second.t);
  }

  void shared(int64_t a, int64_t b, std::vector<int>& ax, std::vector<int>& ay) {
    ax.clear();
    ay.clear();
    const Live& A = live[a];
    const Live& B = live[b];
    for (int k = 0; k < (int)A.ids.size(); ++k) {
      auto it = partner.find(A.ids[k]);
      if (it == partner.end() || owner[it->second] != b) continue;
      const int j = (int)(std::find(B.ids.begin(), B.ids.end(), it->second) - B.ids.begin());
      ax.push_back(k);
      ay.push_back(j);
    }
  }

  std::vector<int64_t> neighbours(int64_t a) {
    std::set<int64_t> s;
    for (int64_t id : live[a].ids) {
      auto it = partner.find(id);
      if (it != partner.end()) s.insert(owner[it->second]);
    }
    return std::vector<int64_t>(s.begin(), s.end());
  }

  int64_t bond_dim(int64_t a, int64_t b) {
    std::vector<int> ax, ay;
    shared(a, b, ax, ay);
    int64_t d = 1;
    for (int k : ax) d *= (int64_t)live[a].t->d0[k] + live[a].t->d1[k];
    return d;
  }

  void set_ids(int64_t i, std::vector<int64_t> ids) {
    for (int64_t id : ids) owner[id] = i;
    live[i].ids = std::move(ids);
  }

  ftn_status init(ftn_ctx ctx, const ftn_network* net, const ftn_tree* tr, ftn_prec pr) {
    if (!net || !tr) return set_error(FTN_EINVAL, "null argument");
    n = net->n_tensors;
    if (n < 1 || !net->tensors) return set_error(FTN_EINVAL, "empty network");
    if (tr->n_steps != n - 1 || (n > 1 && !tr->pairs)) return set_error(FTN_EINVAL, "tree needs n_tensors - 1 steps");
    if (tr->policy != FTN_POLICY_EXACT && tr->chi < 1) return set_error(FTN_EINVAL, "chi must be >= 1");
    if (net->n_bonds > 0 && !net->bonds) return set_error(FTN_EINVAL, "null bond table");
    tree = tr;
    prec = pr;
    global = net->positions != nullptr;
    const ftn_dtype want = prec == FTN_PREC_F64 ? FTN_F64 : FTN_F32;
    for (int i = 0; i < n; ++i) {
      ftn_tensor t = net->tensors[i];
      if (!t) return set_error(FTN_EINVAL, "null tensor in network");
      if (t->dtype != want) return set_error(FTN_EUNSUPPORTED, "tensor dtype does not match the precision");
      ftn_tensor view = nullptr;  // borrowed view: the executor never frees caller buffers
      Live L;
      if (!global && t->parity) {
        // Locally ordered formalism, odd tensor (Sec. II.D): one more leg, odd
        // and of size 1, makes it even.  Appended last, it keeps every
        // nonzero block at the same offset with the same row-major shape, so
        // the view reads the caller's buffer unchanged.
        if (t->rank + 1 > MAXR) return set_error(FTN_EUNSUPPORTED, "odd tensor of maximal rank in the local formalism");
        int32_t d0[MAXR], d1[MAXR];
        uint8_t du[MAXR];
        for (int k = 0; k < t->rank; ++k) d0[k] = t->d0[k], d1[k] = t->d1[k], du[k] = t->dual[k];
        d0[t->rank] = 0, d1[t->rank] = 1, du[t->rank] = 0;
        FTN_TRY(ftn_tensor_wrap(ctx, t->rank + 1, d0, d1, du, 0, t->dtype, t->data, &view));
        dummy[(int64_t)i * 64 + t->rank] = i;
      } else {
        FTN_TRY(ftn_tensor_wrap(ctx, t->rank, t->d0, t->d1, t->dual, t->parity, t->dtype, t->data, &view));
      }
      L.t = view;
      L.pos = global ? net->positions[i] : 0;
      for (int k = 0; k < view->rank; ++k) L.ids.push_back((int64_t)i * 64 + k);
      live[i] = L;
      for (int k = 0; k < view->rank; ++k) owner[(int64_t)i * 64 + k] = i;
    }
    for (int b = 0; b < net->n_bonds; ++b) {
      const int32_t* q = net->bonds + 4 * b;
      if (q[0] < 0 || q[0] >= n || q[2] < 0 || q[2] >= n || q[1] < 0 || q[3] < 0 ||
          q[1] >= net->tensors[q[0]]->rank || q[3] >= net->tensors[q[2]]->rank)
        return set_error(FTN_EINVAL, "bond out of range");
      const int64_t u = (int64_t)q[0] * 64 + q[1], v = (int64_t)q[2] * 64 + q[3];
      if (u == v || partner.count(u) || partner.count(v)) return set_error(FTN_EINVAL, "leg bonded twice");
      partner[u] = v;
      partner[v] = u;
    }
    return FTN_OK;
  }

  // the operands of step s, checked
  ftn_status step_pair(int s, int64_t& a, int64_t& b) {
    a = tree->pairs[2 * s];
    b = tree->pairs[2 * s + 1];
    if (!live.count(a) || !live.count(b) || a == b) return set_error(FTN_EINVAL, "tree refers to a dead tensor");
    return FTN_OK;
  }

  // Compressions before a step (late policy): every other bond of both
  // operands above chi, operand a first, neighbours in increasing id.  A
  // compression changes only the bond it compresses, so the whole list can
  // be taken before the first of them runs.
  std::vector<std::pair<int64_t, int64_t>> late_pairs(int64_t a, int64_t b) {
    std::vector<std::pair<int64_t, int64_t>> out;
    for (int64_t op : {a, b}) {
      const int64_t other = op == a ? b : a;
      for (int64_t nb : neighbours(op))
        if (nb != other && bond_dim(op, nb) > tree->chi) out.push_back({op, nb});
    }
    return out;
  }

  // Compressions after a step (early policy): every bond of the new tensor above chi.
  std::vector<std::pair<int64_t, int64_t>> early_pairs(int64_t id) {
    std::vector<std::pair<int64_t, int64_t>> out;
    for (int64_t nb : neighbours(id))
      if (bond_dim(id, nb) > tree->chi) out.push_back({id, nb});
    return out;
  }

  // The compression of the bond between x and y as a batch item (x becomes
  // the earlier tensor in the global order).
  void compress_item(int64_t& x, int64_t& y, CompressItem& it) {
    if (global && live[x].pos > live[y].pos) std::swap(x, y);
    std::vector<int> ax, ay;
    shared(x, y, ax, ay);
    it.X = live[x].t;
    it.Y = live[y].t;
    it.n = (int)ax.size();
    for (int i = 0; i < it.n; ++i) it.ax[i] = ax[i], it.ay[i] = ay[i];
    it.chi = tree->chi;
    it.arrows = global ? 0 : 1;
  }

  // After the compression: the shared legs of x and y are one new bond (last
  // leg of x, first leg of y).
  void compress_done(int64_t x, int64_t y, const CompressItem& it) {
    Live& X = live[x];
    Live& Y = live[y];
    std::vector<int64_t> fx, fy;
    for (int k = 0; k < (int)X.ids.size(); ++k)
      if (std::find(it.ax, it.ax + it.n, k) == it.ax + it.n) fx.push_back(X.ids[k]);
      else
        partner.erase(X.ids[k]);
    for (int k = 0; k < (int)Y.ids.size(); ++k)
      if (std::find(it.ay, it.ay + it.n, k) == it.ay + it.n) fy.push_back(Y.ids[k]);
      else
        partner.erase(Y.ids[k]);
    const int64_t lx = next_leg++, ly = next_leg++;
    partner[lx] = ly;
    partner[ly] = lx;
    fx.push_back(lx);
    fy.insert(fy.begin(), ly);
    set_ids(x, fx);
    set_ids(y, fy);
  }

  // The pairwise contraction of a step as a batch item: e is the earlier
  // operand, l the later (moved past the tensors between them).
  void step_item(int64_t a, int64_t b, int64_t& e, int64_t& l, TdItem& it) {
    std::vector<int> ax, ay;
    e = a;
    l = b;
    uint64_t flip_e = 0, flip_l = 0;
    if (global) {
      if (live[a].pos > live[b].pos) std::swap(e, l);
      std::vector<int> cx, cl;
      for (auto& kv : live) {
        const int64_t c = kv.first;
        if (c == e || c == l || !(live[e].pos < kv.second.pos && kv.second.pos < live[l].pos)) continue;
        shared(c, l, cx, cl);
        for (int k : cl) flip_l |= 1ull << k;
        if (kv.second.t->parity & live[l].t->parity) sign = -sign;
      }
      shared(e, l, ax, ay);
      for (int k : ax)  // plain ordered contraction: cancel the arrow parity
        if (live[e].t->dual[k] == 0) flip_e |= 1ull << k;
    } else {
      shared(e, l, ax, ay);
    }
    it.A = live[e].t;
    it.B = live[l].t;
    it.n = (int)ax.size();
    for (int i = 0; i < it.n; ++i) it.ax[i] = ax[i], it.ay[i] = ay[i];
    it.fa = flip_e;
    it.fb = flip_l;
    it.C = nullptr;
  }

  // The result of step s replaces its operands (id n + s at e's position).
  int64_t step_done(int s, int64_t e, int64_t l, const TdItem& it) {
    std::vector<int64_t> ids;
    for (int k = 0; k < (int)live[e].ids.size(); ++k)
      if (std::find(it.ax, it.ax + it.n, k) == it.ax + it.n) ids.push_back(live[e].ids[k]);
      else
        partner.erase(live[e].ids[k]);
    for (int k = 0; k < (int)live[l].ids.size(); ++k)
      if (std::find(it.ay, it.ay + it.n, k) == it.ay + it.n) ids.push_back(live[l].ids[k]);
      else
        partner.erase(live[l].ids[k]);
    const int64_t pos = live[e].pos;
    if (retain) {
      retain->push_back(live[e].t);
      retain->push_back(live[l].t);
    } else {
      ftn_tensor_free(live[e].t);
      ftn_tensor_free(live[l].t);
    }
    live.erase(e);
    live.erase(l);
    const int64_t id = n + s;
    Live L;
    L.t = it.C;
    L.pos = pos;
    live[id] = L;
    set_ids(id, ids);
    return id;
  }
};

// Replaces the two tensors of every pair by their cast to `to` (batched).
ftn_status cast_pairs(ftn_ctx ctx, std::vector<Exec*>& nets, std::vector<std::pair<int64_t, int64_t>>& pairs,
                      std::vector<CompressItem>& items, ftn_dtype to) {
  std::vector<ftn_tensor> in, out;
  for (auto& it : items) {
    in.push_back(it.X);
    in.push_back(it.Y);
  }
  FTN_TRY(cast_batch(ctx, in, to, out));
  for (size_t q = 0; q < items.size(); ++q) {
    Live& X = nets[q]->live[pairs[q].first];
    Live& Y = nets[q]->live[pairs[q].second];
    ftn_tensor_free(X.t);
    ftn_tensor_free(Y.t);
    X.t = items[q].X = out[2 * q];
    Y.t = items[q].Y = out[2 * q + 1];
  }
  return FTN_OK;
}

// One sub-round of compressions: pairs[q] of network nets[q].  FP32
// networks compress in FP64 (cast there and back, batched as well).
ftn_status run_compressions(ftn_ctx ctx, std::vector<Exec*>& nets, std::vector<std::pair<int64_t, int64_t>>& pairs) {
  if (nets.empty()) return FTN_OK;
  std::vector<CompressItem> items(nets.size());
  for (size_t q = 0; q < nets.size(); ++q) nets[q]->compress_item(pairs[q].first, pairs[q].second, items[q]);
  const bool f32 = items[0].X->dtype == FTN_F32;
  if (f32) FTN_TRY(cast_pairs(ctx, nets, pairs, items, FTN_F64));  // the decomposition runs in FP64
  // on failure the inputs are untouched and still owned by their networks
  FTN_TRY(compress_batch(ctx, items));
  for (size_t q = 0; q < items.size(); ++q) {
    nets[q]->live[pairs[q].first].t = items[q].X;
    nets[q]->live[pairs[q].second].t = items[q].Y;
  }
  if (f32) FTN_TRY(cast_pairs(ctx, nets, pairs, items, FTN_F32));
  for (size_t q = 0; q < items.size(); ++q) nets[q]->compress_done(pairs[q].first, pairs[q].second, items[q]);
  return FTN_OK;
}

// The compressions of one round in sub-rounds: position j of every network's list.
ftn_status compress_lists(ftn_ctx ctx, std::vector<Exec*>& nets,
                          std::vector<std::vector<std::pair<int64_t, int64_t>>>& lists) {
  size_t depth = 0;
  for (auto& l : lists) depth = std::max(depth, l.size());
  for (size_t j = 0; j < depth; ++j) {
    std::vector<Exec*> sub;
    std::vector<std::pair<int64_t, int64_t>> pairs;
    for (size_t q = 0; q < nets.size(); ++q)
      if (j < lists[q].size()) {
        sub.push_back(nets[q]);
        pairs.push_back(lists[q][j]);
      }
    FTN_TRY(run_compressions(ctx, sub, pairs));
  }
  return FTN_OK;
}

}  // namespace

// Every network walked in lock step; d_out[2 i] = sign x mantissa and
// d_out[2 i + 1] = log-scale of network i, written on the device in stream
// order (no host synchronisation, so the call can be captured into a graph
// when every plan exists and no compression runs).
static ftn_status contract_batch_run(ftn_ctx ctx, int count, const ftn_network* nets, const ftn_tree* trees,
                                     ftn_prec prec, double* d_out) {
  std::vector<std::unique_ptr<Exec>> ex(count);
  int max_steps = 0;
  for (int i = 0; i < count; ++i) {
    ex[i].reset(new Exec());
    FTN_TRY(ex[i]->init(ctx, &nets[i], &trees[i], prec));
    max_steps = std::max(max_steps, ex[i]->n - 1);
  }
  // device scratch per network: [log-scale accumulator, two max |x| words]
  constexpr int STATE = 32;
  void* d_state = dev_alloc(ctx, (size_t)count * STATE + 256);
  if (!d_state) return set_error(FTN_ENOMEM, "device allocation failed");
  struct Guard {
    ftn_ctx c;
    void* p;
    ~Guard() { dev_free(c, p); }
  } guard{ctx, d_state};
  FTN_CUDA(cudaMemsetAsync(d_state, 0, (size_t)count * STATE, ctx->stream));
  auto state = [&](int i) { return (void*)((char*)d_state + (size_t)i * STATE); };
  for (int s = 0; s < max_steps; ++s) {
    std::vector<int> act;
    for (int i = 0; i < count; ++i)
      if (s < ex[i]->n - 1) act.push_back(i);
    std::vector<Exec*> an;
    std::vector<int64_t> a(act.size()), b(act.size());
    for (size_t q = 0; q < act.size(); ++q) {
      an.push_back(ex[act[q]].get());
      FTN_TRY(an[q]->step_pair(s, a[q], b[q]));
    }
    {  // compressions before the step
      std::vector<Exec*> who;
      std::vector<std::vector<std::pair<int64_t, int64_t>>> lists;
      for (size_t q = 0; q < act.size(); ++q)
        if (an[q]->tree->policy == FTN_POLICY_LATE) {
          who.push_back(an[q]);
          lists.push_back(an[q]->late_pairs(a[q], b[q]));
        }
      FTN_TRY(compress_lists(ctx, who, lists));
    }
    // the pairwise contractions
    std::vector<TdItem> items(act.size());
    std::vector<int64_t> e(act.size()), l(act.size()), id(act.size());
    for (size_t q = 0; q < act.size(); ++q) an[q]->step_item(a[q], b[q], e[q], l[q], items[q]);
    FTN_TRY(tensordot_batch(ctx, items, prec));
    for (size_t q = 0; q < act.size(); ++q) id[q] = an[q]->step_done(s, e[q], l[q], items[q]);
    {  // compressions after the step
      std::vector<Exec*> who;
      std::vector<std::vector<std::pair<int64_t, int64_t>>> lists;
      for (size_t q = 0; q < act.size(); ++q)
        if (an[q]->tree->policy == FTN_POLICY_EARLY) {
          who.push_back(an[q]);
          lists.push_back(an[q]->early_pairs(id[q]));
        }
      FTN_TRY(compress_lists(ctx, who, lists));
    }
    std::vector<NormItem> norm;
    for (size_t q = 0; q < act.size(); ++q) norm.push_back({an[q]->live[id[q]].t, state(act[q]), s});
    FTN_TRY(normalize_batch(ctx, norm));
  }
  std::vector<ResultJob> res(count);
  for (int i = 0; i < count; ++i) {
    Exec& E = *ex[i];
    if (E.live.size() != 1) return set_error(FTN_EINVAL, "tree does not reduce the network to one tensor");
    ftn_tensor last = E.live.begin()->second.t;
    // Only the dummy legs of odd tensors may remain (locally ordered
    // formalism); sorting them by decreasing tensor index is a fermionic
    // transposition of odd legs: one sign per inverted pair.
    const std::vector<int64_t>& left = E.live.begin()->second.ids;
    std::vector<int> own;
    for (int64_t id : left) {
      auto it = E.dummy.find(id);
      if (it == E.dummy.end()) return set_error(FTN_EINVAL, "network is not closed (open legs remain)");
      own.push_back(it->second);
    }
    if (own.size() != E.dummy.size()) return set_error(FTN_EINVAL, "internal error: dummy legs lost");
    for (size_t p = 0; p < own.size(); ++p)
      for (size_t q = p + 1; q < own.size(); ++q)
        if (own[p] < own[q]) E.sign = -E.sign;
    res[i].value = last->numel ? last->data : nullptr;
    res[i].logacc = (const double*)state(i);
    res[i].f64 = last->dtype == FTN_F64 ? 1 : 0;
    res[i].sign = E.sign;
  }
  struct Guard2 {
    ftn_ctx c;
    void* p;
    ~Guard2() { dev_free(c, p); }
  } guard2{ctx, nullptr};
  FTN_TRY(upload_table(ctx, res.data(), (size_t)count * sizeof(ResultJob), &guard2.p));
  return launch_gather_results(ctx, (const ResultJob*)guard2.p, count, d_out);
}

ftn_status contract_batch_impl(ftn_ctx ctx, int count, const ftn_network* nets, const ftn_tree* trees, ftn_prec prec,
                               double* mantissa, double* log_scale) {
  if (!ctx || count < 0 || (count > 0 && (!nets || !trees || !mantissa || !log_scale)))
    return set_error(FTN_EINVAL, "null argument");
  if (count == 0) return FTN_OK;
  if (!prec_valid(prec)) return set_error(FTN_EINVAL, "bad precision");
  void* d_out = dev_alloc(ctx, (size_t)count * 16);
  if (!d_out) return set_error(FTN_ENOMEM, "device allocation failed");
  struct Guard {
    ftn_ctx c;
    void* p;
    ~Guard() { dev_free(c, p); }
  } guard{ctx, d_out};
  FTN_TRY(contract_batch_run(ctx, count, nets, trees, prec, (double*)d_out));
  std::vector<double> host(2 * (size_t)count);
  FTN_CUDA(cudaMemcpyAsync(host.data(), d_out, host.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
  FTN_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < count; ++i) {
    mantissa[i] = host[2 * i];
    log_scale[i] = host[2 * i + 1];
  }
  return FTN_OK;
}

ftn_status contract_batch_async_impl(ftn_ctx ctx, int count, const ftn_network* nets, const ftn_tree* trees,
                                     ftn_prec prec, double* d_out) {
  if (!ctx || count < 0 || (count > 0 && (!nets || !trees || !d_out))) return set_error(FTN_EINVAL, "null argument");
  if (count == 0) return FTN_OK;
  if (!prec_valid(prec)) return set_error(FTN_EINVAL, "bad precision");
  return contract_batch_run(ctx, count, nets, trees, prec, d_out);
}

// ---- gradient of a network's value (ftn_contract_grad) ----------------------
// Forward: the executor's walk (same pairs, same late / early compressions of
// the same bonds, same flips and phases) without the per-step normalisation,
// one network, FP64.  Backward: the cotangent of the final scalar is its
// sign; each contraction passes the cotangent of its result to its operands
// by ftn_tensordot_grad (the same flips), each compression the cotangents of
// X', Y' to X, Y by ftn_compress_grad (forward recomputed, same kept set); the
// leaves' cotangents are dv/dT.  Scope: even tensors (no dummy legs), the
// compression's differentiability conditions; the value must stay within
// FP64's range.
//
// Checkpointing (checkpoint = k > 0): the steps are cut into segments of k.
// A first walk keeps only the state at each segment start (its live tensors
// and the executor's bookkeeping) and frees every other intermediate; the
// backward then takes the segments last to first, puts the segment's
// starting state back, replays its steps keeping their operands, and runs
// them backwards.  The cotangents reaching the end of a replayed segment are
// those of the next segment's starting tensors, matched by tensor id: the
// kernels are deterministic, so a replay reproduces the first walk's tensors
// (and kept sets) bit for bit.  Memory: the checkpoints plus one segment's
// operands, for one extra forward pass over all but the last segment.
// checkpoint = 0 is one segment: every operand kept, no replay.
ftn_status contract_grad_impl(ftn_ctx ctx, const ftn_network* net, const ftn_tree* tree, int checkpoint,
                              double* value, ftn_tensor* grads) {
  if (!ctx || !net || !tree || !value || !grads) return set_error(FTN_EINVAL, "null argument");
  if (checkpoint < 0) return set_error(FTN_EINVAL, "checkpoint must be >= 0");
  for (int i = 0; i < net->n_tensors; ++i) grads[i] = nullptr;
  Exec E;
  FTN_TRY(E.init(ctx, net, tree, FTN_PREC_F64));
  for (int i = 0; i < E.n; ++i)
    if (net->tensors[i]->parity) return set_error(FTN_EUNSUPPORTED, "network gradient: even tensors only");
  struct Op {
    bool td;
    ftn_tensor a, b, c, d;  // td: A, B, C; compression: X, Y, X', Y'
    int n;
    int ax[MAXR], ay[MAXR];
    uint64_t fa, fb;
    int chi, arrows;
    CompressState* st;  // compression: its forward, kept for the adjoint (taped walks)
  };
  // Every tensor made here (the leaves' views included) is in `owned` until
  // it is freed, every cotangent in `g`; both are released on every return.
  std::set<ftn_tensor> owned;
  std::map<ftn_tensor, ftn_tensor> g;
  struct Cleanup {
    Exec& e;
    std::set<ftn_tensor>& o;
    std::map<ftn_tensor, ftn_tensor>& g;
    ~Cleanup() {
      e.live.clear();  // owned below, not by the executor
      for (ftn_tensor t : o) ftn_tensor_free(t);
      for (auto& kv : g) ftn_tensor_free(kv.second);
    }
  } cleanup{E, owned, g};
  for (auto& kv : E.live) owned.insert(kv.second.t);
  auto drop = [&](ftn_tensor t) {
    if (owned.erase(t)) ftn_tensor_free(t);
  };
  std::vector<ftn_tensor> consumed;  // operands of the current step (freed or kept by the caller)
  E.retain = &consumed;
  auto compress_pair = [&](int64_t x, int64_t y, std::vector<Op>* tape) -> ftn_status {
    std::vector<CompressItem> items(1);
    E.compress_item(x, y, items[0]);
    items[0].keep_inputs = true;
    Op op{};
    op.td = false;
    op.a = items[0].X;
    op.b = items[0].Y;
    op.n = items[0].n;
    for (int i = 0; i < op.n; ++i) op.ax[i] = items[0].ax[i], op.ay[i] = items[0].ay[i];
    op.chi = items[0].chi;
    op.arrows = items[0].arrows;
    if (tape) items[0].keep_state = &op.st;  // the adjoint reuses this forward instead of recomputing it
    FTN_TRY(compress_batch(ctx, items));
    consumed.push_back(op.a);
    consumed.push_back(op.b);
    op.c = items[0].X;
    op.d = items[0].Y;
    owned.insert(op.c);
    owned.insert(op.d);
    E.live[x].t = op.c;
    E.live[y].t = op.d;
    E.compress_done(x, y, items[0]);
    if (tape) tape->push_back(op);
    return FTN_OK;
  };
  struct TapeStates {  // kept compression states not yet consumed (an early return)
    std::vector<Op>* t = nullptr;
    ~TapeStates() {
      if (t)
        for (Op& o : *t) free_compress_state(o.st);
    }
  };
  auto run_step = [&](int s, std::vector<Op>* tape) -> ftn_status {
    int64_t a, b;
    FTN_TRY(E.step_pair(s, a, b));
    if (tree->policy == FTN_POLICY_LATE)
      for (auto& pr : E.late_pairs(a, b)) FTN_TRY(compress_pair(pr.first, pr.second, tape));
    std::vector<TdItem> items(1);
    int64_t e, l;
    E.step_item(a, b, e, l, items[0]);
    FTN_TRY(tensordot_batch(ctx, items, FTN_PREC_F64));
    owned.insert(items[0].C);
    if (tape) {
      Op op{};
      op.td = true;
      op.a = items[0].A;
      op.b = items[0].B;
      op.c = items[0].C;
      op.n = items[0].n;
      for (int i = 0; i < op.n; ++i) op.ax[i] = items[0].ax[i], op.ay[i] = items[0].ay[i];
      op.fa = items[0].fa;
      op.fb = items[0].fb;
      tape->push_back(op);
    }
    const int64_t id = E.step_done(s, e, l, items[0]);
    if (tree->policy == FTN_POLICY_EARLY)
      for (auto& pr : E.early_pairs(id)) FTN_TRY(compress_pair(pr.first, pr.second, tape));
    return FTN_OK;
  };
  const int S = E.n - 1;
  const int k = (checkpoint == 0 || checkpoint >= S) ? std::max(S, 1) : checkpoint;
  const int J = S <= 0 ? 1 : (S + k - 1) / k;
  std::vector<Exec::State> snaps(J);
  std::set<ftn_tensor> pinned;  // the checkpoints' tensors (kept until the end)
  std::vector<ftn_tensor> leaves(E.n);  // the executor's views of the caller's tensors
  for (int i = 0; i < E.n; ++i) leaves[i] = E.live[i].t;
  E.save(snaps[0]);
  for (auto& kv : E.live) pinned.insert(kv.second.t);
  // first walk: up to the last checkpoint, keeping only the checkpoints
  for (int s = 0; s < (J - 1) * k; ++s) {
    FTN_TRY(run_step(s, nullptr));
    for (ftn_tensor t : consumed)
      if (!pinned.count(t)) drop(t);
    consumed.clear();
    if ((s + 1) % k == 0) {
      E.save(snaps[(s + 1) / k]);
      for (auto& kv : E.live) pinned.insert(kv.second.t);
    }
  }
  auto cot = [&](ftn_tensor t, ftn_tensor* out) -> ftn_status {  // the cotangent of t (zeros if none reached it)
    auto it = g.find(t);
    if (it != g.end()) {
      *out = it->second;
      return FTN_OK;
    }
    ftn_tensor z = nullptr;
    FTN_TRY(make_tensor(ctx, t->rank, t->d0, t->d1, t->dual, t->parity, FTN_F64, &z));
    g[t] = z;
    FTN_CUDA(cudaMemsetAsync(z->data, 0, (size_t)z->numel * 8, ctx->stream));
    *out = z;
    return FTN_OK;
  };
  auto put = [&](ftn_tensor t, ftn_tensor d) -> ftn_status {
    if (g.count(t)) {
      ftn_tensor_free(d);
      return set_error(FTN_EINVAL, "internal error: a tensor of the tape is consumed twice");
    }
    g[t] = d;
    return FTN_OK;
  };
  auto release = [&](ftn_tensor t) {  // a cotangent that has been passed on
    auto it = g.find(t);
    if (it == g.end()) return;
    ftn_tensor_free(it->second);
    g.erase(it);
  };
  for (int j = J - 1; j >= 0; --j) {
    // replay segment j from its checkpoint, keeping its operands
    E.load(snaps[j]);
    std::vector<Op> tape;
    TapeStates tape_states;
    tape_states.t = &tape;
    consumed.clear();
    const int s_end = std::min(S, (j + 1) * k);
    for (int s = j * k; s < s_end; ++s) FTN_TRY(run_step(s, &tape));
    if (j == J - 1) {
      if (E.live.size() != 1) return set_error(FTN_EINVAL, "tree does not reduce the network to one tensor");
      ftn_tensor last = E.live.begin()->second.t;
      if (last->numel != 1) return set_error(FTN_EINVAL, "network is not closed (open legs remain)");
      double v = 0.0;
      FTN_CUDA(cudaMemcpyAsync(&v, last->data, 8, cudaMemcpyDeviceToHost, ctx->stream));
      FTN_CUDA(cudaStreamSynchronize(ctx->stream));
      *value = E.sign * v;
      // seed: dv/d(last) = sign
      ftn_tensor seed = nullptr;
      FTN_TRY(make_tensor(ctx, last->rank, last->d0, last->d1, last->dual, last->parity, FTN_F64, &seed));
      g[last] = seed;
      const double sg = (double)E.sign;
      FTN_CUDA(cudaMemcpyAsync(seed->data, &sg, 8, cudaMemcpyHostToDevice, ctx->stream));
      FTN_CUDA(cudaStreamSynchronize(ctx->stream));  // the host source goes out of scope
    } else {
      // the replayed end state is checkpoint j + 1: its tensors take the
      // cotangents of that checkpoint's (same ids, same values)
      if (E.live.size() != snaps[j + 1].live.size())
        return set_error(FTN_EINVAL, "internal error: a replayed segment ends in another state");
      for (auto& kv : E.live) {
        auto sn = snaps[j + 1].live.find(kv.first);
        if (sn == snaps[j + 1].live.end())
          return set_error(FTN_EINVAL, "internal error: a replayed segment ends in another state");
        const ftn_tensor ts = sn->second.t, tr = kv.second.t;
        if (ts == tr) continue;
        auto it = g.find(ts);
        if (it == g.end()) continue;
        const ftn_tensor d = it->second;
        g.erase(it);
        FTN_TRY(put(tr, d));
      }
    }
    for (auto it = tape.rbegin(); it != tape.rend(); ++it) {
      Op& op = *it;
      if (op.td) {
        ftn_tensor G = nullptr, dA = nullptr, dB = nullptr;
        FTN_TRY(cot(op.c, &G));
        FTN_TRY(ftn_tensordot_grad(ctx, op.a, op.b, G, op.n, op.ax, op.ay, op.fa, op.fb, nullptr, FTN_PREC_F64, &dA,
                                   &dB));
        release(op.c);
        FTN_TRY(put(op.a, dA));
        FTN_TRY(put(op.b, dB));
      } else {
        ftn_tensor gx = nullptr, gy = nullptr, dX = nullptr, dY = nullptr;
        FTN_TRY(cot(op.c, &gx));
        FTN_TRY(cot(op.d, &gy));
        if (op.st) {
          FTN_TRY(compress_backward(ctx, op.st, gx, gy, &dX, &dY));
          free_compress_state(op.st);
          op.st = nullptr;
        } else {
          FTN_TRY(ftn_compress_grad(ctx, op.a, op.b, op.n, op.ax, op.ay, op.chi, op.arrows, gx, gy, &dX, &dY));
        }
        release(op.c);
        release(op.d);
        FTN_TRY(put(op.a, dX));
        FTN_TRY(put(op.b, dY));
      }
    }
    // the segment's tensors, but for the checkpoints', are no longer needed
    for (ftn_tensor t : consumed)
      if (!pinned.count(t)) drop(t);
    consumed.clear();
    for (auto& kv : E.live)
      if (!pinned.count(kv.second.t)) drop(kv.second.t);
    E.live.clear();
  }
  // the leaves' cotangents (the views have the caller's legs)
  for (int i = 0; i < E.n; ++i) {
    ftn_tensor d = nullptr;
    if (leaves[i]) {
      auto f = g.find(leaves[i]);
      if (f != g.end()) {
        d = f->second;
        g.erase(f);
      }
    }
    if (!d) {  // a tensor whose value does not reach the result (cannot happen in a connected tree)
      FTN_TRY(make_tensor(ctx, net->tensors[i]->rank, net->tensors[i]->d0, net->tensors[i]->d1,
                          net->tensors[i]->dual, 0, FTN_F64, &d));
      FTN_CUDA(cudaMemsetAsync(d->data, 0, (size_t)d->numel * 8, ctx->stream));
    }
    grads[i] = d;
  }
  return FTN_OK;
}

ftn_status contract_impl(ftn_ctx ctx, const ftn_network* net, const ftn_tree* tree, ftn_prec prec, double* mantissa,
                         double* log_scale) {
  if (!ctx || !net || !tree || !mantissa || !log_scale) return set_error(FTN_EINVAL, "null argument");
  return contract_batch_impl(ctx, 1, net, tree, prec, mantissa, log_scale);
}

// ---- Hubbard operator tensors ---------------------------------------------------
namespace {

// local state -> (n_up, n_dn): 0 = |0>, 1 = |up dn>, 2 = |up>, 3 = |dn>
const int OCC[4][2] = {{0, 0}, {1, 1}, {1, 0}, {0, 1}};

// Fermionic mode operators on occupation bit strings, modes ordered
// (i up, i dn, j up, j dn); the sign counts occupied modes before the mode.
bool apply_annihilate(int mode, unsigned& state, int& sign) {
  if (!((state >> mode) & 1u)) return false;
  for (int k = 0; k < mode; ++k)
    if ((state >> k) & 1u) sign = -sign;
  state &= ~(1u << mode);
  return true;
}
bool apply_create(int mode, unsigned& state, int& sign) {
  if ((state >> mode) & 1u) return false;
  for (int k = 0; k < mode; ++k)
    if ((state >> k) & 1u) sign = -sign;
  state |= 1u << mode;
  return true;
}

unsigned pack(int si, int sj) {
  return (unsigned)(OCC[si][0] | (OCC[si][1] << 1) | (OCC[sj][0] << 2) | (OCC[sj][1] << 3));
}

}  // namespace

ftn_status hubbard_impl(ftn_ctx ctx, int kind, double t, double u, ftn_dtype dtype, ftn_tensor* out) {
  if (!ctx || !out) return set_error(FTN_EINVAL, "null argument");
  if (kind != 0 && kind != 1) return set_error(FTN_EINVAL, "kind must be 0 (hopping) or 1 (on-site)");
  const int r = kind == 0 ? 4 : 2;
  int32_t d0[4] = {2, 2, 2, 2}, d1[4] = {2, 2, 2, 2};
  uint8_t du[4] = {0, 0, 1, 1};
  if (kind == 1) du[1] = 1;
  ftn_tensor T = nullptr;
  FTN_TRY(make_tensor(ctx, r, d0, d1, du, 0, dtype, &T));
  std::vector<double> dense(r == 4 ? 256 : 16, 0.0);
  if (kind == 0) {
    // O[n_i, n_j, m_j, m_i] = <n_i n_j| -t sum_s (c+_is c_js + c+_js c_is) |m_i m_j>
    for (int mi = 0; mi < 4; ++mi)
      for (int mj = 0; mj < 4; ++mj)
        for (int s = 0; s < 2; ++s)
          for (int dir = 0; dir < 2; ++dir) {
            const int from = dir == 0 ? 2 + s : s;  // annihilated mode
            const int to = dir == 0 ? s : 2 + s;    // created mode
            unsigned st = pack(mi, mj);
            int sg = 1;
            if (!apply_annihilate(from, st, sg) || !apply_create(to, st, sg)) continue;
            int ni = -1, nj = -1;
            for (int a = 0; a < 4; ++a)
              for (int b = 0; b < 4; ++b)
                if (pack(a, b) == st) ni = a, nj = b;
            dense[((ni * 4 + nj) * 4 + mj) * 4 + mi] += -t * sg;
          }
  } else {
    dense[1 * 4 + 1] = u;  // U n_up n_dn on |up dn>
  }
  // pack into the block layout: dense index 0,1 even (sector-local 0,1), 2,3 odd
  std::vector<double> packed(T->numel);
  for (int64_t b = 0; b < nblocks(r, 0); ++b) {
    const uint32_t m = block_mask(r, 0, b);
    int64_t off = T->offsets[b];
    const int nel = 1 << r;  // 2 per leg
    for (int e = 0; e < nel; ++e) {
      int idx = 0;
      for (int k = 0; k < r; ++k) {
        const int loc = (e >> (r - 1 - k)) & 1;  // row-major over legs
        idx = idx * 4 + (((m >> k) & 1) ? 2 + loc : loc);
      }
      packed[off + e] = dense[idx];
    }
  }
  if (dtype == FTN_F64) {
    FTN_CUDA(cudaMemcpyAsync(T->data, packed.data(), packed.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    FTN_CUDA(cudaStreamSynchronize(ctx->stream));
  } else {
    std::vector<float> p32(packed.begin(), packed.end());
    FTN_CUDA(cudaMemcpyAsync(T->data, p32.data(), p32.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    FTN_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  *out = T;
  return FTN_OK;
}

}  // namespace ftn

using namespace ftn;

extern "C" {

ftn_status ftn_contract(ftn_ctx ctx, const ftn_network* net, const ftn_tree* tree, ftn_prec prec, double* mantissa,
                        double* log_scale) {
  return contract_impl(ctx, net, tree, prec, mantissa, log_scale);
}

ftn_status ftn_contract_grad(ftn_ctx ctx, const ftn_network* net, const ftn_tree* tree, int checkpoint,
                             double* value, ftn_tensor* grads) {
  return contract_grad_impl(ctx, net, tree, checkpoint, value, grads);
}

ftn_status ftn_contract_batch(ftn_ctx ctx, int count, const ftn_network* nets, const ftn_tree* trees, ftn_prec prec,
                              double* mantissa, double* log_scale) {
  return contract_batch_impl(ctx, count, nets, trees, prec, mantissa, log_scale);
}

ftn_status ftn_contract_batch_async(ftn_ctx ctx, int count, const ftn_network* nets, const ftn_tree* trees,
                                    ftn_prec prec, double* d_out) {
  return contract_batch_async_impl(ctx, count, nets, trees, prec, d_out);
}

ftn_status ftn_hubbard_term(ftn_ctx ctx, int kind, double t, double u, ftn_dtype dtype, ftn_tensor* out) {
  return hubbard_impl(ctx, kind, t, u, dtype, out);
}

}  // extern "C"
