// Contraction-tree executor ftn_contract (Fig. 1; Secs. II.C-II.D; Sec. III)
// and the Hubbard operator tensors ftn_hubbard_term (Eq. fermi-hubbard-ham).
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
#include <algorithm>
#include <cmath>
#include <map>
#include <set>

#include "tdplan.h"

namespace ftn {

ftn_status normalize_tensor(ftn_ctx ctx, ftn_tensor t, void* d_state, int step);
ftn_status cast_tensor(ftn_ctx ctx, ftn_tensor t, ftn_dtype to, ftn_tensor* out);
ftn_status compress_impl(ftn_ctx ctx, ftn_tensor* pX, ftn_tensor* pY, int n, const int* ax, const int* ay, int chi,
                         int arrows, ftn_compress_info* info);
ftn_status tensordot_impl(ftn_ctx ctx, ftn_tensor A, ftn_tensor B, int n, const int* ax, const int* ay,
                          uint64_t flip_a, uint64_t flip_b, const int* out_perm, ftn_prec prec, ftn_tensor* C);

namespace {

struct Live {
  ftn_tensor t = nullptr;
  std::vector<int64_t> ids;  // leg identities
  int64_t pos = 0;
};

struct Exec {
  ftn_ctx ctx;
  ftn_prec prec;
  bool global = false;
  std::map<int64_t, Live> live;
  std::map<int64_t, int64_t> partner;  // leg id -> leg id
  std::map<int64_t, int64_t> owner;    // leg id -> tensor id
  int64_t next_leg = 1ll << 40;
  int sign = 1;
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

  ftn_status compress_pair(int64_t x, int64_t y, int chi) {
    if (global && live[x].pos > live[y].pos) std::swap(x, y);
    std::vector<int> ax, ay;
    shared(x, y, ax, ay);
    Live& X = live[x];
    Live& Y = live[y];
    ftn_tensor tx = X.t, ty = Y.t;
    const bool f32 = tx->dtype == FTN_F32;
    if (f32) {  // the decomposition runs in FP64
      ftn_tensor wx = nullptr, wy = nullptr;
      FTN_TRY(cast_tensor(ctx, tx, FTN_F64, &wx));
      ftn_status st = cast_tensor(ctx, ty, FTN_F64, &wy);
      if (st != FTN_OK) {
        ftn_tensor_free(wx);
        return st;
      }
      ftn_tensor_free(tx);
      ftn_tensor_free(ty);
      tx = wx;
      ty = wy;
      X.t = tx;
      Y.t = ty;
    }
    FTN_TRY(compress_impl(ctx, &tx, &ty, (int)ax.size(), ax.data(), ay.data(), chi, global ? 0 : 1, nullptr));
    X.t = tx;
    Y.t = ty;
    if (f32) {
      ftn_tensor nx = nullptr, ny = nullptr;
      FTN_TRY(cast_tensor(ctx, tx, FTN_F32, &nx));
      FTN_TRY(cast_tensor(ctx, ty, FTN_F32, &ny));
      ftn_tensor_free(tx);
      ftn_tensor_free(ty);
      X.t = nx;
      Y.t = ny;
    }
    std::vector<int64_t> fx, fy;
    for (int k = 0; k < (int)X.ids.size(); ++k)
      if (std::find(ax.begin(), ax.end(), k) == ax.end()) fx.push_back(X.ids[k]);
      else
        partner.erase(X.ids[k]);
    for (int k = 0; k < (int)Y.ids.size(); ++k)
      if (std::find(ay.begin(), ay.end(), k) == ay.end()) fy.push_back(Y.ids[k]);
      else
        partner.erase(Y.ids[k]);
    const int64_t lx = next_leg++, ly = next_leg++;
    partner[lx] = ly;
    partner[ly] = lx;
    fx.push_back(lx);
    fy.insert(fy.begin(), ly);
    set_ids(x, fx);
    set_ids(y, fy);
    return FTN_OK;
  }
};

}  // namespace

ftn_status contract_impl(ftn_ctx ctx, const ftn_network* net, const ftn_tree* tree, ftn_prec prec, double* mantissa,
                         double* log_scale) {
  if (!ctx || !net || !tree || !mantissa || !log_scale) return set_error(FTN_EINVAL, "null argument");
  const int n = net->n_tensors;
  if (n < 1 || !net->tensors) return set_error(FTN_EINVAL, "empty network");
  if (tree->n_steps != n - 1 || (n > 1 && !tree->pairs)) return set_error(FTN_EINVAL, "tree needs n_tensors - 1 steps");
  if (tree->policy != FTN_POLICY_EXACT && tree->chi < 1) return set_error(FTN_EINVAL, "chi must be >= 1");
  const ftn_dtype want = prec == FTN_PREC_F64 ? FTN_F64 : FTN_F32;
  Exec E;
  E.ctx = ctx;
  E.prec = prec;
  E.global = net->positions != nullptr;
  for (int i = 0; i < n; ++i) {
    ftn_tensor t = net->tensors[i];
    if (!t) return set_error(FTN_EINVAL, "null tensor in network");
    if (t->dtype != want) return set_error(FTN_EUNSUPPORTED, "tensor dtype does not match the precision");
    ftn_tensor view = nullptr;  // borrowed view: the executor never frees caller buffers
    FTN_TRY(ftn_tensor_wrap(ctx, t->rank, t->d0, t->d1, t->dual, t->parity, t->dtype, t->data, &view));
    Live L;
    L.t = view;
    L.pos = E.global ? net->positions[i] : 0;
    for (int k = 0; k < t->rank; ++k) L.ids.push_back((int64_t)i * 64 + k);
    E.live[i] = L;
    for (int k = 0; k < t->rank; ++k) E.owner[(int64_t)i * 64 + k] = i;
  }
  for (int b = 0; b < net->n_bonds; ++b) {
    const int32_t* q = net->bonds + 4 * b;
    if (q[0] < 0 || q[0] >= n || q[2] < 0 || q[2] >= n || q[1] < 0 || q[3] < 0 ||
        q[1] >= net->tensors[q[0]]->rank || q[3] >= net->tensors[q[2]]->rank)
      return set_error(FTN_EINVAL, "bond out of range");
    const int64_t u = (int64_t)q[0] * 64 + q[1], v = (int64_t)q[2] * 64 + q[3];
    if (E.partner.count(u) || E.partner.count(v)) return set_error(FTN_EINVAL, "leg bonded twice");
    E.partner[u] = v;
    E.partner[v] = u;
  }
  // device scratch: [log-scale accumulator, two max |x| words]
  void* d_state = dev_alloc(ctx, 256);
  if (!d_state) return set_error(FTN_ENOMEM, "device allocation failed");
  struct Guard {
    ftn_ctx c;
    void* p;
    ~Guard() { dev_free(c, p); }
  } guard{ctx, d_state};
  FTN_CUDA(cudaMemsetAsync(d_state, 0, 24, ctx->stream));
  const int chi = tree->chi;
  for (int s = 0; s < n - 1; ++s) {
    const int64_t a = tree->pairs[2 * s], b = tree->pairs[2 * s + 1];
    if (!E.live.count(a) || !E.live.count(b) || a == b) return set_error(FTN_EINVAL, "tree refers to a dead tensor");
    if (tree->policy == FTN_POLICY_LATE) {
      for (int64_t op : {a, b}) {
        const int64_t other = op == a ? b : a;
        for (int64_t nb : E.neighbours(op))
          if (nb != other && E.bond_dim(op, nb) > chi) FTN_TRY(E.compress_pair(op, nb, chi));
      }
    }
    std::vector<int> ax, ay;
    int64_t e = a, l = b;
    uint64_t flip_e = 0, flip_l = 0;
    if (E.global) {
      if (E.live[a].pos > E.live[b].pos) std::swap(e, l);
      // move l leftwards past every tensor between the two positions
      std::vector<int> cx, cl;
      for (auto& kv : E.live) {
        const int64_t c = kv.first;
        if (c == e || c == l || !(E.live[e].pos < kv.second.pos && kv.second.pos < E.live[l].pos)) continue;
        E.shared(c, l, cx, cl);
        for (int k : cl) flip_l |= 1ull << k;
        if (kv.second.t->parity & E.live[l].t->parity) E.sign = -E.sign;
      }
      E.shared(e, l, ax, ay);
      for (int k : ax)  // plain ordered contraction: cancel the arrow parity
        if (E.live[e].t->dual[k] == 0) flip_e |= 1ull << k;
    } else {
      E.shared(e, l, ax, ay);
    }
    ftn_tensor C = nullptr;
    FTN_TRY(tensordot_impl(ctx, E.live[e].t, E.live[l].t, (int)ax.size(), ax.data(), ay.data(), flip_e, flip_l,
                           nullptr, prec, &C));
    std::vector<int64_t> ids;
    for (int k = 0; k < (int)E.live[e].ids.size(); ++k)
      if (std::find(ax.begin(), ax.end(), k) == ax.end()) ids.push_back(E.live[e].ids[k]);
      else
        E.partner.erase(E.live[e].ids[k]);
    for (int k = 0; k < (int)E.live[l].ids.size(); ++k)
      if (std::find(ay.begin(), ay.end(), k) == ay.end()) ids.push_back(E.live[l].ids[k]);
      else
        E.partner.erase(E.live[l].ids[k]);
    const int64_t pos = E.live[e].pos;
    ftn_tensor_free(E.live[e].t);
    ftn_tensor_free(E.live[l].t);
    E.live.erase(e);
    E.live.erase(l);
    const int64_t id = n + s;
    Live L;
    L.t = C;
    L.pos = pos;
    E.live[id] = L;
    E.set_ids(id, ids);
    if (tree->policy == FTN_POLICY_EARLY)
      for (int64_t nb : E.neighbours(id))
        if (E.bond_dim(id, nb) > chi) FTN_TRY(E.compress_pair(id, nb, chi));
    FTN_TRY(normalize_tensor(ctx, E.live[id].t, d_state, s));
  }
  if (E.live.size() != 1) return set_error(FTN_EINVAL, "tree does not reduce the network to one tensor");
  ftn_tensor last = E.live.begin()->second.t;
  if (last->rank != 0) return set_error(FTN_EINVAL, "network is not closed (open legs remain)");
  double host_state[2] = {0, 0};
  double val = 0.0;
  FTN_CUDA(cudaMemcpyAsync(host_state, d_state, 16, cudaMemcpyDeviceToHost, ctx->stream));
  if (last->numel) {
    if (last->dtype == FTN_F64) {
      FTN_CUDA(cudaMemcpyAsync(&val, last->data, 8, cudaMemcpyDeviceToHost, ctx->stream));
      FTN_CUDA(cudaStreamSynchronize(ctx->stream));
    } else {
      float v32 = 0.f;
      FTN_CUDA(cudaMemcpyAsync(&v32, last->data, 4, cudaMemcpyDeviceToHost, ctx->stream));
      FTN_CUDA(cudaStreamSynchronize(ctx->stream));
      val = v32;
    }
  } else {
    FTN_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  *mantissa = val * E.sign;
  *log_scale = host_state[0];
  return FTN_OK;
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

ftn_status ftn_hubbard_term(ftn_ctx ctx, int kind, double t, double u, ftn_dtype dtype, ftn_tensor* out) {
  return hubbard_impl(ctx, kind, t, u, dtype, out);
}

}  // extern "C"
