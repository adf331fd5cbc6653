"""Dense FP64 graded tensors and the pairwise fermionic operations.

Test infrastructure only (see the package docstring).

Leg convention: ``(d_even, d_odd, dual)``; ``dual = 1`` marks an incoming
('-') leg, ``dual = 0`` an outgoing ('+') leg (Sec. II.A, symmetry rule).  A
bond's arrow runs from its '+' leg to its '-' leg; by default it points from
the later tensor to the earlier one (Sec. IV.B).
"""
from __future__ import annotations

import itertools

import numpy as np

__all__ = [
    "GTensor",
    "index_parity",
    "embed_blocks",
    "extract_blocks",
    "transpose",
    "flip_legs",
    "contract",
    "trace_pair",
    "dagger",
    "contract_outer_literal",
]


def index_parity(d0, d1):
    """Parity of each dense index of a leg: even indices first."""
    return np.concatenate([np.zeros(d0, np.int64), np.ones(d1, np.int64)])


def _bcast(vec, axis, ndim):
    shp = [1] * ndim
    shp[axis] = vec.shape[0]
    return vec.reshape(shp)


class GTensor:
    """A dense-embedded Z2-graded fermionic tensor with definite parity.

    Sec. II.B: a fermionic tensor carries a parity per index, a definite total
    parity and a definite leg order.
    """

    __slots__ = ("data", "legs", "parity")

    def __init__(self, data, legs, parity):
        self.data = np.asarray(data, dtype=np.float64)
        self.legs = [(int(a), int(b), int(c)) for a, b, c in legs]
        self.parity = int(parity) & 1
        want = tuple(a + b for a, b, _ in self.legs)
        if self.data.shape != want:
            raise ValueError(f"shape {self.data.shape} != legs {want}")

    @property
    def rank(self):
        return len(self.legs)

    def parity_field(self):
        """Total parity (mod 2) of every dense index tuple."""
        tot = np.zeros(self.data.shape, np.int64)
        for k, (d0, d1, _) in enumerate(self.legs):
            tot = tot + _bcast(index_parity(d0, d1), k, self.rank)
        return tot & 1

    def check_symmetry(self, atol=0.0):
        """Entries whose index parities do not sum to the tensor parity vanish
        (Eq. symmetryrule with H = 2)."""
        bad = self.parity_field() != self.parity
        return float(np.max(np.abs(self.data[bad]), initial=0.0)) <= atol

    def copy(self):
        return GTensor(self.data.copy(), list(self.legs), self.parity)


def embed_blocks(legs, parity, blocks):
    """Dense tensor from ``[(bits, array), ...]`` blocks (bits: per-leg sector)."""
    shape = tuple(a + b for a, b, _ in legs)
    out = np.zeros(shape, np.float64)
    for bits, arr in blocks:
        if sum(bits) % 2 != parity:
            raise ValueError("block parity does not match the tensor parity")
        sl = tuple(slice(d0, d0 + d1) if b else slice(0, d0) for (d0, d1, _), b in zip(legs, bits))
        out[sl] = arr
    return GTensor(out, legs, parity)


def extract_blocks(t):
    """Inverse of :func:`embed_blocks`: dict bits -> dense block (copies)."""
    out = {}
    for bits in itertools.product((0, 1), repeat=t.rank):
        if sum(bits) % 2 != t.parity:
            continue
        sl = tuple(slice(d0, d0 + d1) if b else slice(0, d0) for (d0, d1, _), b in zip(t.legs, bits))
        out[bits] = t.data[sl].copy()
    return out


def transpose(t, perm):
    """Fermionic transposition to leg order ``perm`` (out leg u = in leg perm[u]).

    Eq. (transposition): swapping two legs i, j multiplies by (-1)^{p_i p_j}.
    A general permutation is a product of such swaps, so every pair of legs
    whose relative order is inverted contributes (-1)^{p_a p_b}.
    """
    perm = [int(p) for p in perm]
    r = t.rank
    if sorted(perm) != list(range(r)):
        raise ValueError("not a permutation")
    data = np.transpose(t.data, perm)
    legs = [t.legs[p] for p in perm]
    expo = np.zeros((1,) * r, np.int64)
    for u in range(r):
        for v in range(u + 1, r):
            if perm[u] > perm[v]:
                pu = _bcast(index_parity(*legs[u][:2]), u, r)
                pv = _bcast(index_parity(*legs[v][:2]), v, r)
                expo = expo + pu * pv
    sign = 1.0 - 2.0 * (expo & 1)
    return GTensor(data * sign, legs, t.parity)


def flip_legs(t, legs_to_flip):
    """Multiply by the bond parity (-1)^{p} on each listed leg (the diagonal
    part of g, Eq. swapeq)."""
    data = t.data
    for k in legs_to_flip:
        d0, d1, _ = t.legs[k]
        data = data * _bcast(1.0 - 2.0 * index_parity(d0, d1), k, t.rank)
    return GTensor(data, list(t.legs), t.parity)


def _check_pairs(x, y, ax, ay, need_opposite=True):
    if len(ax) != len(ay) or len(set(ax)) != len(ax) or len(set(ay)) != len(ay):
        raise ValueError("bad axes")
    for a, b in zip(ax, ay):
        lx, ly = x.legs[a], y.legs[b]
        if lx[:2] != ly[:2]:
            raise ValueError(f"contracted legs differ in sector dims: {lx} vs {ly}")
        if need_opposite and lx[2] == ly[2]:
            raise ValueError("contracted legs must have opposite duals")


def contract(x, y, ax, ay, arrows=True, flip_x=(), flip_y=()):
    """Pairwise fermionic contraction op(X, Y) over leg pairs (ax[i], ay[i]).

    Eq. (standardcontract): X's contracted legs are moved to its end (in the
    order ax), Y's to its front in mirror order (so that ax[-1] meets ay[-1]
    first), each move a fermionic transposition; then a plain sum.  With
    ``arrows`` (locally ordered formalism, Eq. fermionictn2) a pair whose X leg
    is outgoing ('+', the bond's arrow leaves X) is contracted against its
    arrow and picks up the bond parity (-1)^p.  ``arrows=False`` is the plain
    ordered contraction F(XY) of the global formalism.  ``flip_x``/``flip_y``
    list extra legs carrying a bond parity tensor g.  Output legs: X's free
    legs in order, then Y's.
    """
    ax = [int(a) for a in ax]
    ay = [int(a) for a in ay]
    _check_pairs(x, y, ax, ay)
    if flip_x:
        x = flip_legs(x, flip_x)
    if flip_y:
        y = flip_legs(y, flip_y)
    if arrows:
        against = [a for a in ax if x.legs[a][2] == 0]
        if against:
            x = flip_legs(x, against)
    n = len(ax)
    fx = [k for k in range(x.rank) if k not in ax]
    fy = [k for k in range(y.rank) if k not in ay]
    xt = transpose(x, fx + ax)
    yt = transpose(y, list(reversed(ay)) + fy)
    data = np.tensordot(xt.data, yt.data, axes=(list(range(len(fx), x.rank)), list(range(n - 1, -1, -1))))
    legs = [x.legs[k] for k in fx] + [y.legs[k] for k in fy]
    return GTensor(data, legs, x.parity ^ y.parity)


def trace_pair(t, a, b, arrows=True):
    """Fermionic partial trace of legs a < b of one tensor.

    Leg b is moved next to leg a (a fermionic transposition) and the adjacent
    pair is summed; with ``arrows`` the pair picks up (-1)^p when leg a is
    outgoing, exactly as in :func:`contract`.
    """
    if not a < b:
        raise ValueError("need a < b")
    la, lb = t.legs[a], t.legs[b]
    if la[:2] != lb[:2] or la[2] == lb[2]:
        raise ValueError("traced legs must match with opposite duals")
    if arrows and la[2] == 0:
        t = flip_legs(t, [a])
    order = [k for k in range(t.rank) if k != b]
    order.insert(order.index(a) + 1, b)
    tt = transpose(t, order)
    pos = order.index(a)
    data = np.trace(tt.data, axis1=pos, axis2=pos + 1)
    legs = [t.legs[k] for k in order if k not in (a, b)]
    return GTensor(data, legs, t.parity)


def dagger(t):
    """Hermitian conjugate of one tensor: leg order reversed, duals flipped,
    complex conjugate, no extra sign (Sec. II.C: transposing a network reverses
    the tensor order and the indices of every tensor)."""
    data = np.conj(np.transpose(t.data, list(range(t.rank - 1, -1, -1))))
    legs = [(d0, d1, 1 - du) for (d0, d1, du) in reversed(t.legs)]
    return GTensor(np.real_if_close(data), legs, t.parity)


def contract_outer_literal(x, y, ax, ay, arrows=True):
    """Literal definition for tiny inputs: outer product X (x) Y with X's legs
    first and no sign; then, pair by pair, fermionic-transpose Y's leg right
    after X's partner and trace the adjacent pair (bond parity when X's leg is
    outgoing).  Used only as an independent check of :func:`contract`."""
    _check_pairs(x, y, ax, ay)
    t = GTensor(np.multiply.outer(x.data, y.data), x.legs + y.legs, x.parity ^ y.parity)
    ids = [("x", k) for k in range(x.rank)] + [("y", k) for k in range(y.rank)]
    for a, b in zip(ax, ay):
        ia, ib = ids.index(("x", a)), ids.index(("y", b))
        t = trace_pair(t, ia, ib, arrows=arrows)
        ids = [v for v in ids if v not in (("x", a), ("y", b))]
    return t
