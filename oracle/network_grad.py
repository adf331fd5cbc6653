"""Gradient of a closed network's value through the contraction tree and its
compressions (the value of :func:`oracle.network.contract_tree`, locally or
globally ordered formalism, Sec. II.C, Sec. II.D and Sec. III).

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

In the globally ordered formalism the later tensor of a pair is first
multiplied by the bond parity on the legs it passes and by the phase of the
odd tensors it passes (Sec. II.C); both are +-1 per entry, so their adjoint
is the same multiplication, applied here to the cotangent.

Scope: even tensors, no per-step normalisation (the plain value), the
compression's differentiability conditions of
:mod:`oracle.compress_adjoint`.
"""
from __future__ import annotations

import numpy as np

from .adjoint import contract_grad
from .compress import compress
from .compress_adjoint import compress_grad
from .graded import GTensor, contract, flip_legs
from .network import _State, _bond_dim

__all__ = ["contract_tree_grad"]


def _zero_like(t):
    return GTensor(np.zeros(t.data.shape), t.legs, t.parity)


def contract_tree_grad(net, tree, policy="exact", chi=None, mode="local"):
    """(v, [dv/dT_i for every input tensor], min relative gap) for the closed
    network ``net`` contracted along ``tree`` in the locally or globally
    ordered formalism (``mode``, as in :func:`oracle.network.contract_tree`)
    with the given compression policy.  The last item is the smallest gap at a
    truncation cut relative to the largest singular value of that
    compression (None without truncation): finite differences are only
    meaningful while it is not tiny."""
    if any(t.parity for t in net.tensors):
        raise ValueError("even tensors only")
    if mode == "global" and net.positions is None:
        raise ValueError("global mode needs positions")
    glob = mode == "global"
    st = _State(net)
    n = len(net.tensors)
    nodes = list(net.tensors)          # every tensor value, in order of creation
    cur = {i: i for i in range(n)}     # live tensor id -> node
    tape = []
    gaps = []

    def do_compress(x, y):
        if glob and st.pos[x] > st.pos[y]:
            x, y = y, x
        ax, ay = st.shared(x, y)
        tx, ty = nodes[cur[x]], nodes[cur[y]]
        xn, yn, info = compress(tx, ty, ax, ay, chi, arrows=not glob)
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
        tape.append(("compress", cur[x], cur[y], ax, ay, len(nodes) - 2, len(nodes) - 1, not glob))
        cur[x], cur[y] = len(nodes) - 2, len(nodes) - 1

    for s, (a, b) in enumerate(tree):
        a, b = int(a), int(b)
        if policy == "late":
            for op, other in ((a, b), (b, a)):
                for nb in st.neighbours(op):
                    if nb != other and _bond_dim(st, op, nb) > chi:
                        do_compress(op, nb)
        if not glob:
            ax, ay = st.shared(a, b)
            tn = contract(nodes[cur[a]], nodes[cur[b]], ax, ay, arrows=True)
            ids = [lid for k, lid in enumerate(st.ids[a]) if k not in ax] + [
                lid for k, lid in enumerate(st.ids[b]) if k not in ay
            ]
            nodes.append(tn)
            tape.append(("contract", cur[a], cur[b], ax, ay, len(nodes) - 1, True))
            newpos = None
        else:
            e, l = (a, b) if st.pos[a] < st.pos[b] else (b, a)
            ex, ly = st.shared(e, l)
            flips = []
            phase = 0
            for c in list(cur):
                if c in (e, l) or not (st.pos[e] < st.pos[c] < st.pos[l]):
                    continue
                cx, cl = st.shared(c, l)
                flips.extend(cl)
                phase ^= nodes[cur[c]].parity & nodes[cur[l]].parity
            tl = nodes[cur[l]]
            if flips or phase:
                d = flip_legs(tl, flips).data if flips else tl.data
                tl = GTensor(-d if phase else d, tl.legs, tl.parity)
                nodes.append(tl)
                tape.append(("sign", cur[l], flips, phase, len(nodes) - 1))
                il = len(nodes) - 1
            else:
                il = cur[l]
            tn = contract(nodes[cur[e]], tl, ex, ly, arrows=False)
            ids = [lid for k, lid in enumerate(st.ids[e]) if k not in ex] + [
                lid for k, lid in enumerate(st.ids[l]) if k not in ly
            ]
            nodes.append(tn)
            tape.append(("contract", cur[e], il, ex, ly, len(nodes) - 1, False))
            newpos = st.pos[e]
        for x in (a, b):
            del st.t[x]
            del st.ids[x]
            del cur[x]
            st.pos.pop(x, None)
        new = n + s
        st.set(new, tn, ids)
        cur[new] = len(nodes) - 1
        if newpos is not None:
            st.pos[new] = newpos
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
        if rec[0] == "sign":
            _, isrc, flips, phase, iout = rec
            g = adj.pop(iout, None)
            if g is None:
                continue
            d = flip_legs(g, flips).data if flips else g.data
            pairs = ((isrc, GTensor(-d if phase else d, g.legs, g.parity)),)
        elif rec[0] == "contract":
            _, ix, iy, ax, ay, iz, arrows = rec
            g = adj.pop(iz, None)
            if g is None:
                continue
            gx = contract_grad(nodes[ix], nodes[iy], ax, ay, g, wrt="x", arrows=arrows)
            gy = contract_grad(nodes[ix], nodes[iy], ax, ay, g, wrt="y", arrows=arrows)
            pairs = ((ix, gx), (iy, gy))
        else:
            _, ix, iy, ax, ay, kx, ky, arrows = rec
            g_x = adj.pop(kx, None)
            g_y = adj.pop(ky, None)
            if g_x is None and g_y is None:
                continue
            g_x = g_x if g_x is not None else _zero_like(nodes[kx])
            g_y = g_y if g_y is not None else _zero_like(nodes[ky])
            gx, gy = compress_grad(nodes[ix], nodes[iy], ax, ay, chi, g_x, g_y, arrows=arrows)
            pairs = ((ix, gx), (iy, gy))
        for i, gi in pairs:
            prev = adj.get(i)
            adj[i] = gi if prev is None else GTensor(prev.data + gi.data, gi.legs, gi.parity)
    grads = [adj.get(i, _zero_like(net.tensors[i])) for i in range(n)]
    return value, grads, (min(gaps) if gaps else None)
