"""U(1) x parity structure of fermionic tensors (Sec. II.B).

TEST INFRASTRUCTURE ONLY (see the package docstring).

A fermionic tensor may carry a U(1) symmetry besides parity (fermion number
for the Hubbard model): every index has an integer charge, the parity of a
charge is the charge mod 2, and the fermionic signs depend on the parity
alone.  A U(1)-symmetric tensor is therefore a Z2-graded tensor of the same
dense embedding whose nonzero entries also conserve the charge, and every
Z2 operation of :mod:`oracle.graded` applies to it unchanged.

A U(1) leg is ``(sectors, dual)`` with ``sectors = [(charge, dim), ...]``.
Its Z2 leg is ``(d_even, d_odd, dual)``: the even-charge sectors first, in
the listed order, then the odd ones (the even-first index convention).  An
entry of a tensor of total charge Q is allowed when
sum_k s_k q_k(i_k) = Q, with s_k = +1 on an outgoing leg (dual 0) and -1 on
an incoming leg (dual 1); the tensor's parity is Q mod 2.  A bond pairs two
legs with the same sectors and opposite duals, so its charges cancel and a
contraction has total charge Q_X + Q_Y.
"""
from __future__ import annotations

import numpy as np

from .graded import GTensor

__all__ = ["u1_leg", "u1_z2_legs", "u1_mask", "random_u1", "u1_violation", "u1_result_legs", "HUBBARD_SITE"]

# the physical leg of a Hubbard site in the oracle's index order
# (0 = |0>, 1 = |up dn>, 2 = |up>, 3 = |dn>): fermion numbers 0, 2, 1, 1
HUBBARD_SITE = [(0, 1), (2, 1), (1, 2)]


def u1_leg(sectors, dual):
    """(Z2 leg, charge of every dense index) of a U(1) leg."""
    even = [(q, d) for q, d in sectors if q % 2 == 0]
    odd = [(q, d) for q, d in sectors if q % 2 != 0]
    charges = [q for q, d in even for _ in range(d)] + [q for q, d in odd for _ in range(d)]
    d0 = sum(d for _, d in even)
    d1 = sum(d for _, d in odd)
    return (d0, d1, int(dual)), np.array(charges, dtype=np.int64)


def u1_z2_legs(legs_u1):
    return [u1_leg(s, du)[0] for s, du in legs_u1]


def u1_mask(legs_u1, total):
    """Allowed entries (dense shape) of a U(1) tensor of total charge ``total``."""
    r = len(legs_u1)
    tot = np.zeros([1] * r, np.int64)
    for k, (s, du) in enumerate(legs_u1):
        _, q = u1_leg(s, du)
        shp = [1] * r
        shp[k] = len(q)
        tot = tot + (1 if du == 0 else -1) * q.reshape(shp)
    shape = tuple(len(u1_leg(s, du)[1]) for s, du in legs_u1)
    return np.broadcast_to(tot, shape) == total


def random_u1(legs_u1, total, seed):
    """N(0, 1) entries on the allowed set, zeros elsewhere, as a GTensor."""
    mask = u1_mask(legs_u1, total)
    data = np.where(mask, np.random.default_rng(seed).standard_normal(mask.shape), 0.0)
    return GTensor(data, u1_z2_legs(legs_u1), int(total) % 2)


def u1_violation(t, legs_u1, total):
    """Largest |entry| outside the allowed set (0 for a U(1)-symmetric tensor)."""
    mask = u1_mask(legs_u1, total)
    return float(np.max(np.abs(np.where(mask, 0.0, t.data)), initial=0.0))


def u1_result_legs(lx, ly, ax, ay):
    """U(1) legs of op(X, Y): X's free legs in order, then Y's; the paired
    legs must have the same sectors and opposite duals."""
    for a, b in zip(ax, ay):
        if list(lx[a][0]) != list(ly[b][0]) or lx[a][1] == ly[b][1]:
            raise ValueError("paired U(1) legs must have the same sectors and opposite duals")
    return [lx[k] for k in range(len(lx)) if k not in ax] + [ly[k] for k in range(len(ly)) if k not in ay]
