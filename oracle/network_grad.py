"""Gradient of a closed network's value through the contraction tree and its
compressions (the value of :func:`oracle.network.contract_tree`, locally
ordered formalism, Sec. II.D and Sec. III).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The tree is walked exactly as :func:`oracle.network.contract_tree` walks it
(same pair order, same late/early compressions of the same bonds, neighbours
in increasing id), recording every pairwise contraction and every
compression on a tape with the tensors it consumed.  The value v of the
closed network is then differentiated in reverse order of the tape: a
contraction passes the cotangent of its result to its operands by the
contraction adjoint (:func:`oracle.adjoint.contract_grad`, by definition) and a
compression passes the cotangents of X' and Y' to X and Y by the compression
adjoint (:func:`oracle.compress_adjoint.compress_grad`).  Returned: v and
dv/dT for every input tensor T (tensors of the network are independent
inputs; a bra that is the dagger of a ket is a separate input here).

Scope: even tensors, no per-step normalisation (the plain value), the
compression's differentiability conditions of
:mod:`oracle.compress_adjoint`.
"""
from __future__ import annotations

import numpy as np

from .adjoint import contract_grad
from .compress import compress
from .compress_adjoint import compress_grad
from .graded import GTensor, contract
from .network import _State, _bond_dim

__all__ = ["contract_tree_grad"]


def _zero_like(t):
    return GTensor(np.zeros(t.data.shape), t.legs, t.parity)


def contract_tree_grad(net, tree, policy="exact", chi=None):
    """(v, [dv/dT_i for every input tensor], min relative gap) for the closed
    network ``net`` contracted along ``tree`` (locally ordered formalism) with
    the given compression policy.  The last item is the smallest gap at a
    truncation cut relative to the largest singular value of that
    compression (None without truncation): finite differences are only
    meaningful while it is not tiny."""
    if any(t.parity for t in net.tensors):
        raise ValueError("even tensors only")
    st = _State(net)
    n = len(net.tensors)
    nodes = list(net.tensors)          # every tensor value, in order of creation
    cur = {i: i for i in range(n)}     # live tensor id -> node
    tape = []
    gaps = []

    def do_compress(x, y):
        ax, ay = st.shared(x, y)
        tx, ty = nodes[cur[x]], nodes[cur[y]]
        xn, yn, info = compress(tx, ty, ax, ay, chi, arrows=True)
        if info["gap"] is not None and info["singular_values"]:
            gaps.append(info["gap"] / info["singular_values"][0])
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
        nodes.extend([xn, yn])
        tape.append(("compress", cur[x], cur[y], ax, ay, len(nodes) - 2, len(nodes) - 1))
        cur[x], cur[y] = len(nodes) - 2, len(nodes) - 1

    for s, (a, b) in enumerate(tree):
        a, b = int(a), int(b)
        if policy == "late":
            for op, other in ((a, b), (b, a)):
                for nb in st.neighbours(op):
                    if nb != other and _bond_dim(st, op, nb) > chi:
                        do_compress(op, nb)
        ax, ay = st.shared(a, b)
        tn = contract(nodes[cur[a]], nodes[cur[b]], ax, ay, arrows=True)
        ids = [lid for k, lid in enumerate(st.ids[a]) if k not in ax] + [
            lid for k, lid in enumerate(st.ids[b]) if k not in ay
        ]
        nodes.append(tn)
        tape.append(("contract", cur[a], cur[b], ax, ay, len(nodes) - 1))
        for x in (a, b):
            del st.t[x]
            del st.ids[x]
            del cur[x]
        new = n + s
        st.set(new, tn, ids)
        cur[new] = len(nodes) - 1
        if policy == "early":
            for nb in st.neighbours(new):
                if _bond_dim(st, new, nb) > chi:
                    do_compress(new, nb)
    (last,) = list(cur)
    out = nodes[cur[last]]
    if out.rank != 0:
        raise ValueError("the network is not closed")
    value = float(out.data)
    adj = {cur[last]: GTensor(np.ones(()), out.legs, out.parity)}
    for rec in reversed(tape):
        if rec[0] == "contract":
            _, ix, iy, ax, ay, iz = rec
            g = adj.pop(iz, None)
            if g is None:
                continue
            gx = contract_grad(nodes[ix], nodes[iy], ax, ay, g, wrt="x")
            gy = contract_grad(nodes[ix], nodes[iy], ax, ay, g, wrt="y")
        else:
            _, ix, iy, ax, ay, kx, ky = rec
            g_x = adj.pop(kx, None)
            g_y = adj.pop(ky, None)
            if g_x is None and g_y is None:
                continue
            g_x = g_x if g_x is not None else _zero_like(nodes[kx])
            g_y = g_y if g_y is not None else _zero_like(nodes[ky])
            gx, gy = compress_grad(nodes[ix], nodes[iy], ax, ay, chi, g_x, g_y)
        for i, gi in ((ix, gx), (iy, gy)):
            prev = adj.get(i)
            adj[i] = gi if prev is None else GTensor(prev.data + gi.data, gi.legs, gi.parity)
    grads = [adj.get(i, _zero_like(net.tensors[i])) for i in range(n)]
    return value, grads, (min(gaps) if gaps else None)
