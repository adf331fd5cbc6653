"""Adjoint (gradient) of the pairwise fermionic contraction, by its definition.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The contraction C = op(X, Y) of :func:`oracle.graded.contract` (Eq.
standardcontract with the arrow rule of Eq. fermionictn2), followed by an
optional fermionic transposition of the result (Eq. transposition), is linear
in each operand.  For a scalar L = sum(G * C) the gradient with respect to X
is therefore, entry by entry over the parity-allowed entries i of X,

    dL/dX[i] = sum(G * C(E_i)),

with E_i the graded tensor of X's legs and parity that is 1 at entry i and 0
elsewhere.  That sum is computed here literally, one contraction per entry
(small tensors only); the same for Y.
"""
from __future__ import annotations

import itertools

import numpy as np

from .graded import GTensor, contract, index_parity, transpose

__all__ = ["contract_forward", "contract_grad"]


def contract_forward(x, y, ax, ay, arrows=True, flip_x=(), flip_y=(), out_perm=None):
    """op(X, Y) then, if given, the fermionic transposition out_perm."""
    c = contract(x, y, ax, ay, arrows=arrows, flip_x=flip_x, flip_y=flip_y)
    if out_perm is not None:
        c = transpose(c, list(out_perm))
    return c


def _allowed(t):
    """Indices of the parity-allowed entries of a graded tensor."""
    par = [index_parity(d0, d1) for d0, d1, _ in t.legs]
    for idx in itertools.product(*[range(len(p)) for p in par]):
        if sum(int(par[k][i]) for k, i in enumerate(idx)) % 2 == t.parity:
            yield idx


def contract_grad(x, y, ax, ay, g, wrt="x", arrows=True, flip_x=(), flip_y=(), out_perm=None):
    """dL/dX (wrt="x") or dL/dY (wrt="y") for L = sum(G * C), C as in
    :func:`contract_forward`; G has C's legs and parity.  Returns a GTensor
    with the differentiated operand's legs and parity."""
    t = x if wrt == "x" else y
    out = np.zeros(t.data.shape)
    for idx in _allowed(t):
        e = np.zeros(t.data.shape)
        e[idx] = 1.0
        et = GTensor(e, t.legs, t.parity)
        c = contract_forward(et, y, ax, ay, arrows, flip_x, flip_y, out_perm) if wrt == "x" else \
            contract_forward(x, et, ax, ay, arrows, flip_x, flip_y, out_perm)
        out[idx] = float(np.sum(g.data * c.data))
    return GTensor(out, t.legs, t.parity)
