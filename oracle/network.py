"""Fermionic tensor networks: tree executor (local and global formalisms) and
brute-force evaluation of the globally ordered value.

Test infrastructure only (see the package docstring).

A network is a list of :class:`~oracle.graded.GTensor` plus bonds
``(t1, leg1, t2, leg2)``.  Global positions, when given, are the integer
order of the tensors in F(A^[0] B^[1] ...) (Eq. fermionictn).
"""
from __future__ import annotations

import math

import numpy as np

from .graded import GTensor, contract, flip_legs, index_parity, transpose
from .compress import compress

__all__ = ["Network", "contract_tree", "brute_force_global", "arrows_from_positions"]


class Network:
    def __init__(self, tensors, bonds, positions=None):
        self.tensors = list(tensors)
        self.bonds = [tuple(int(v) for v in b) for b in bonds]
        self.positions = None if positions is None else [int(p) for p in positions]
        seen = set()
        for t1, l1, t2, l2 in self.bonds:
            for key in ((t1, l1), (t2, l2)):
                if key in seen:
                    raise ValueError(f"leg {key} bonded twice")
                seen.add(key)
            a, b = self.tensors[t1].legs[l1], self.tensors[t2].legs[l2]
            if a[:2] != b[:2] or a[2] == b[2]:
                raise ValueError(f"bond {(t1, l1, t2, l2)} has mismatched legs {a} {b}")


def arrows_from_positions(net):
    """True when every bond's '-' leg sits on the earlier tensor, i.e. the
    arrows (from '+' to '-') point from later to earlier tensors (Sec. IV.B),
    so that the bonds form the DAG of the global order (Sec. II.C)."""
    for t1, l1, t2, l2 in net.bonds:
        early, el = (t1, l1) if net.positions[t1] < net.positions[t2] else (t2, l2)
        if net.tensors[early].legs[el][2] != 1:
            return False
    return True


class _State:
    def __init__(self, net):
        self.t = {}
        self.ids = {}
        self.partner = {}
        self.pos = {}
        self.owner = {}
        for i, tn in enumerate(net.tensors):
            self.t[i] = tn
            self.ids[i] = [(i, k) for k in range(tn.rank)]
            for k in range(tn.rank):
                self.owner[(i, k)] = i
            if net.positions is not None:
                self.pos[i] = net.positions[i]
        for t1, l1, t2, l2 in net.bonds:
            self.partner[(t1, l1)] = (t2, l2)
            self.partner[(t2, l2)] = (t1, l1)
        self.new_leg = 0

    def shared(self, a, b):
        ax, ay = [], []
        for k, lid in enumerate(self.ids[a]):
            p = self.partner.get(lid)
            if p is not None and self.owner[p] == b:
                ax.append(k)
                ay.append(self.ids[b].index(p))
        return ax, ay

    def neighbours(self, a):
        out = set()
        for lid in self.ids[a]:
            p = self.partner.get(lid)
            if p is not None:
                out.add(self.owner[p])
        return sorted(out)

    def set(self, i, tn, ids):
        self.t[i] = tn
        self.ids[i] = ids
        for lid in ids:
            self.owner[lid] = i


def _bond_dim(st, a, b):
    ax, _ = st.shared(a, b)
    return math.prod(st.t[a].legs[k][0] + st.t[a].legs[k][1] for k in ax)


def _compress_pair(st, x, y, chi, mode):
    """Compress the bond between live tensors x and y (all shared legs fused)."""
    if mode == "global" and st.pos[x] > st.pos[y]:
        x, y = y, x
    ax, ay = st.shared(x, y)
    xn, yn, _info = compress(st.t[x], st.t[y], ax, ay, chi, arrows=(mode == "local"))
    fx = [lid for k, lid in enumerate(st.ids[x]) if k not in ax]
    fy = [lid for k, lid in enumerate(st.ids[y]) if k not in ay]
    st.new_leg += 1
    lx, ly = ("c", st.new_leg, 0), ("c", st.new_leg, 1)
    for k in ax:
        st.partner.pop(st.ids[x][k], None)
    for k in ay:
        st.partner.pop(st.ids[y][k], None)
    st.partner[lx], st.partner[ly] = ly, lx
    st.set(x, xn, fx + [lx])
    st.set(y, yn, [ly] + fy)


def contract_tree(net, tree, mode="local", policy="exact", chi=None, normalize=False):
    """Walk an SSA contraction tree (Fig. 1) and return (tensor, log_scale, leg ids).

    ``mode='local'``: pairwise contractions with the bond parity applied when a
    bond is contracted against its arrow (Eq. fermionictn2); odd tensors are
    made even with a dummy leg (see :func:`_contract_local_odd`).
    ``mode='global'``: the later tensor of each pair is first moved leftwards
    past every tensor between the two positions; each shared bond it passes
    carries a bond parity g and each odd tensor it passes a phase
    (-1)^{p_b p_c} (Sec. II.C); then the plain ordered contraction F(ab) runs.
    ``policy``: 'exact', 'early' or 'late' compression of bonds whose
    dimension exceeds ``chi`` (Sec. III): late compresses the other bonds of
    both operands just before they are contracted, early compresses the bonds
    of each new tensor right after it is formed; neighbours are visited in
    increasing tensor id.  ``normalize`` divides every new tensor by its
    largest |entry| and accumulates the natural log of the factors.
    """
    if mode == "global" and net.positions is None:
        raise ValueError("global mode needs positions")
    odd = [i for i, t in enumerate(net.tensors) if t.parity] if mode == "local" else []
    if odd:
        return _contract_local_odd(net, tree, policy, chi, normalize, odd)
    st = _State(net)
    n = len(net.tensors)
    log_scale = 0.0
    for s, (a, b) in enumerate(tree):
        a, b = int(a), int(b)
        if policy == "late":
            for op, other in ((a, b), (b, a)):
                for nb in st.neighbours(op):
                    if nb != other and _bond_dim(st, op, nb) > chi:
                        _compress_pair(st, op, nb, chi, mode)
        ax, ay = st.shared(a, b)
        if mode == "local":
            tn = contract(st.t[a], st.t[b], ax, ay, arrows=True)
            ids = [lid for k, lid in enumerate(st.ids[a]) if k not in ax] + [
                lid for k, lid in enumerate(st.ids[b]) if k not in ay
            ]
            newpos = None
        else:
            e, l = (a, b) if st.pos[a] < st.pos[b] else (b, a)
            ex, ly = st.shared(e, l)
            flips = []
            phase = 0
            for c in list(st.t):
                if c in (e, l) or not (st.pos[e] < st.pos[c] < st.pos[l]):
                    continue
                cx, cl = st.shared(c, l)
                flips.extend(cl)
                phase ^= st.t[c].parity & st.t[l].parity
            tl = flip_legs(st.t[l], flips) if flips else st.t[l]
            tn = contract(st.t[e], tl, ex, ly, arrows=False)
            if phase:
                tn = GTensor(-tn.data, tn.legs, tn.parity)
            ids = [lid for k, lid in enumerate(st.ids[e]) if k not in ex] + [
                lid for k, lid in enumerate(st.ids[l]) if k not in ly
            ]
            newpos = st.pos[e]
        for x in (a, b):
            del st.t[x]
            del st.ids[x]
            st.pos.pop(x, None)
        new = n + s
        st.set(new, tn, ids)
        if newpos is not None:
            st.pos[new] = newpos
        if policy == "early":
            for nb in st.neighbours(new):
                if _bond_dim(st, new, nb) > chi:
                    _compress_pair(st, new, nb, chi, mode)
        if normalize:
            m = float(np.max(np.abs(st.t[new].data), initial=0.0))
            if m > 0:
                st.t[new] = GTensor(st.t[new].data / m, st.t[new].legs, st.t[new].parity)
                log_scale += math.log(m)
    (last,) = list(st.t)
    return st.t[last], log_scale, st.ids[last]


# Order of the dummy legs of odd tensors after a locally ordered contraction
# (see _contract_local_odd).
DUMMY_ORDER_DESCENDING = True


def _contract_local_odd(net, tree, policy, chi, normalize, odd):
    """Locally ordered formalism with odd tensors (Sec. II.D): every odd
    tensor gets one more leg, odd and of size 1, which makes it even; the
    network is contracted as an even one, the dummy legs stay open, and the
    dummy legs left on the result are sorted by decreasing tensor index (a
    fermionic transposition, so each exchange of two of them is a sign).
    The value is that of the globally ordered network with the tensors in
    index order (reading of the ordering convention, pinned in the tests
    against the brute-force global value)."""
    tensors = list(net.tensors)
    for i in odd:
        t = tensors[i]
        tensors[i] = GTensor(t.data[..., None], list(t.legs) + [(0, 1, 0)], 0)
    inner = Network(tensors, net.bonds, None)
    res, log_scale, ids = contract_tree(inner, tree, mode="local", policy=policy, chi=chi, normalize=normalize)
    owners = [tk[0] for tk in ids]
    if sorted(owners) != sorted(odd):
        raise ValueError("network is not closed")
    order = sorted(range(len(ids)), key=lambda q: owners[q], reverse=DUMMY_ORDER_DESCENDING)
    if len(order) > 1:
        res = transpose(res, order)
    val = res.data.reshape(-1)[0] if res.data.size else 0.0
    return GTensor(np.array(val), [], 0), log_scale, []


def brute_force_global(net):
    """Value of a closed network F(T^[0] T^[1] ...) by an explicit sum over every
    assignment of bond indices.

    The literal definition of the ordered contraction: the legs of all tensors
    are laid out in position order; each term carries the sign of the
    permutation (restricted to odd legs) that brings every bond's later leg
    right behind its earlier leg (Eq. transposition applied to the whole
    string); no arrow signs enter F (Eq. fermionictn).
    """
    order = sorted(range(len(net.tensors)), key=lambda i: net.positions[i])
    slot = {}
    seq = []
    for t in order:
        for k in range(net.tensors[t].rank):
            slot[(t, k)] = len(seq)
            seq.append((t, k))
    if len(net.bonds) * 2 != len(seq):
        raise ValueError("network is not closed")
    pairs = []
    for t1, l1, t2, l2 in net.bonds:
        u, v = slot[(t1, l1)], slot[(t2, l2)]
        pairs.append((min(u, v), max(u, v)))
    pairs.sort()
    target = np.empty(len(seq), np.int64)
    for q, (u, v) in enumerate(pairs):
        target[u] = 2 * q
        target[v] = 2 * q + 1
    bond_of_slot = {}
    for q, (u, v) in enumerate(pairs):
        bond_of_slot[u] = q
        bond_of_slot[v] = q
    dims = []
    dpar = []
    for u, v in pairs:
        t, k = seq[u]
        d0, d1, _ = net.tensors[t].legs[k]
        dims.append(d0 + d1)
        dpar.append(index_parity(d0, d1))
    grids = np.meshgrid(*[np.arange(d) for d in dims], indexing="ij")
    assign = np.stack([g.reshape(-1) for g in grids], axis=1)  # (n_terms, n_bonds)
    par = np.stack([dpar[q][assign[:, q]] for q in range(len(pairs))], axis=1)
    slot_par = par[:, [bond_of_slot[s] for s in range(len(seq))]]
    expo = np.zeros(assign.shape[0], np.int64)
    for a in range(len(seq)):
        for b in range(a + 1, len(seq)):
            if target[a] > target[b]:
                expo += slot_par[:, a] * slot_par[:, b]
    val = 1.0 - 2.0 * (expo & 1)
    for t in order:
        tn = net.tensors[t]
        idx = tuple(assign[:, bond_of_slot[slot[(t, k)]]] for k in range(tn.rank))
        val = val * tn.data[idx]
    return float(np.sum(val))

