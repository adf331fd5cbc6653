"""Sector-wise QR/SVD bond compression (Sec. II.A, Sec. II.B, Sec. III).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from .graded import GTensor, _check_pairs, flip_legs, index_parity, transpose

__all__ = ["compress", "matricize_pair", "transpose_sign_at", "contract_sampled"]


def _multi_parity(legs):
    """Parity of every row-major multi-index over ``legs`` (flattened)."""
    if not legs:
        return np.zeros(1, np.int64)
    tot = np.zeros([a + b for a, b, _ in legs], np.int64)
    r = len(legs)
    for k, (d0, d1, _) in enumerate(legs):
        shp = [1] * r
        shp[k] = d0 + d1
        tot = tot + index_parity(d0, d1).reshape(shp)
    return (tot & 1).reshape(-1)


def matricize_pair(x, y, ax, ay, arrows=True):
    """Fermionic-transpose X to [free | bond] and Y to [bond (mirror) | free] and
    return the two matrices whose plain product is op(X, Y) (Sec. II.B: the
    decomposition runs after transposing into row | column order), plus the
    free leg lists and the row/bond/column parities."""
    ax = [int(a) for a in ax]
    ay = [int(a) for a in ay]
    _check_pairs(x, y, ax, ay)
    if arrows:
        against = [a for a in ax if x.legs[a][2] == 0]
        if against:
            x = flip_legs(x, against)
    n = len(ax)
    fx = [k for k in range(x.rank) if k not in ax]
    fy = [k for k in range(y.rank) if k not in ay]
    xt = transpose(x, fx + ax)
    yt = transpose(y, list(reversed(ay)) + fy)
    rdims = [x.legs[k][0] + x.legs[k][1] for k in fx]
    bdims = [x.legs[k][0] + x.legs[k][1] for k in ax]
    cdims = [y.legs[k][0] + y.legs[k][1] for k in fy]
    R, K, C = int(np.prod(rdims)), int(np.prod(bdims)), int(np.prod(cdims))
    xm = xt.data.reshape(R, K)
    # plain (sign-free) reordering of the mirrored bond axes back to ax order
    ydata = np.transpose(yt.data, list(range(n - 1, -1, -1)) + list(range(n, yt.rank)))
    ym = ydata.reshape(K, C)
    rpar = _multi_parity([x.legs[k] for k in fx])
    kpar = _multi_parity([x.legs[k] for k in ax])
    cpar = _multi_parity([y.legs[k] for k in fy])
    return xm, ym, fx, fy, rpar, kpar, cpar


def compress(x, y, ax, ay, chi, arrows=True):
    """Compress the bond (legs ax of X paired with ay of Y) to at most chi.

    Steps, in the order of the paper's symmetric decompositions (Sec. II.A):
    per bond-parity sector pi, QR of X_pi = Q_X R_X and of Y_pi^T = Q_Y R_Y; SVD
    of the core M_pi = R_X R_Y^T; the singular values of all sectors are pooled
    and the chi largest kept (ties: lower sector, then lower index); then
    X' = Q_X U sqrt(S) and Y' = sqrt(S) V^T Q_Y^T.  Q keeps the parity of its
    tensor (s(Q) = s(A), s(U) = s(A)), so R, M and S are even.

    Returns (X', Y', info).  X' has X's free legs in order then the new leg
    (incoming, '-'); Y' has the new leg (outgoing, '+') then Y's free legs, so
    that op(X', Y') is sign-free and approximates op(X, Y).
    """
    xm, ym, fx, fy, rpar, kpar, cpar = matricize_pair(x, y, ax, ay, arrows=arrows)
    px, py = x.parity, y.parity
    sec = {}
    cand = []
    for pi in (0, 1):
        rows = np.nonzero(rpar == (px ^ pi))[0]
        ks = np.nonzero(kpar == pi)[0]
        cols = np.nonzero(cpar == (py ^ pi))[0]
        sec[pi] = (rows, ks, cols)
        if len(rows) == 0 or len(ks) == 0 or len(cols) == 0:
            sec[pi] += (None,)
            continue
        xp = xm[np.ix_(rows, ks)]
        yp = ym[np.ix_(ks, cols)]
        qx, rx = np.linalg.qr(xp)
        qy, ry = np.linalg.qr(yp.T)
        u, s, vt = np.linalg.svd(rx @ ry.T, full_matrices=False)
        sec[pi] += ((qx, qy, u, s, vt),)
        for i, sv in enumerate(s):
            cand.append((-float(sv), pi, i))
    cand.sort()
    kept = cand[: max(int(chi), 0)]
    k = [sum(1 for c in kept if c[1] == pi) for pi in (0, 1)]
    discarded = float(sum(c[0] ** 2 for c in cand[len(kept):]))
    R, C = xm.shape[0], ym.shape[1]
    xnew = np.zeros((R, k[0] + k[1]))
    ynew = np.zeros((k[0] + k[1], C))
    off = {0: 0, 1: k[0]}
    for pi in (0, 1):
        rows, ks, cols, fac = sec[pi]
        if fac is None or k[pi] == 0:
            continue
        qx, qy, u, s, vt = fac
        kk = k[pi]
        rs = np.sqrt(s[:kk])
        xnew[np.ix_(rows, np.arange(off[pi], off[pi] + kk))] = (qx @ u[:, :kk]) * rs
        ynew[np.ix_(np.arange(off[pi], off[pi] + kk), cols)] = (rs[:, None] * vt[:kk]) @ qy.T
    xlegs = [x.legs[q] for q in fx] + [(k[0], k[1], 1)]
    ylegs = [(k[0], k[1], 0)] + [y.legs[q] for q in fy]
    xs = tuple(a + b for a, b, _ in xlegs)
    ys = tuple(a + b for a, b, _ in ylegs)
    allsv = sorted((-c[0] for c in cand), reverse=True)
    gap = None
    if len(kept) < len(cand) and kept:
        gap = -kept[-1][0] - (-cand[len(kept)][0])
    info = {
        "kept": tuple(k),
        "discarded_sq": discarded,
        "singular_values": allsv,
        "sector_sv": {pi: (None if sec[pi][3] is None else sec[pi][3][3]) for pi in (0, 1)},
        "gap": gap,
    }
    return GTensor(xnew.reshape(xs), xlegs, px), GTensor(ynew.reshape(ys), ylegs, py), info


def transpose_sign_at(legs, perm, index):
    """Sign of Eq. (transposition) for one dense index tuple ``index`` of the
    *input* legs when permuted to out leg u = in leg perm[u]."""
    par = [int(index[k] >= legs[k][0]) for k in range(len(legs))]
    s = 0
    r = len(perm)
    for u in range(r):
        for v in range(u + 1, r):
            if perm[u] > perm[v]:
                s ^= par[perm[u]] & par[perm[v]]
    return -1.0 if s else 1.0


def contract_sampled(x, y, ax, ay, out_perm, n_samples, seed, arrows=True):
    """Selected entries of transpose(op(X, Y), out_perm), each computed as one
    row of [free | bond] X times one column of [bond | free] Y (the
    matricisation of Eq. standardcontract) times the transposition sign.

    Returns (indices into the permuted result, values)."""
    xm, ym, fx, fy, _, _, _ = matricize_pair(x, y, ax, ay, arrows=arrows)
    legs = [x.legs[k] for k in fx] + [y.legs[k] for k in fy]
    dims = [a + b for a, b, _ in legs]
    nfx = len(fx)
    r = len(legs)
    perm = list(range(r)) if out_perm is None else [int(p) for p in out_perm]
    g = np.random.Generator(np.random.PCG64(seed))
    idx_out = []
    vals = []
    total_par = x.parity ^ y.parity
    if n_samples > 0 and not np.any((_multi_parity(legs) & 1) == total_par):
        raise ValueError("the result has no parity-allowed entry to sample")
    while len(vals) < n_samples:
        idx = [int(g.integers(d)) for d in dims]
        if sum(int(idx[k] >= legs[k][0]) for k in range(r)) % 2 != total_par:
            continue  # structurally zero entry; sample allowed ones only
        row = int(np.ravel_multi_index(idx[:nfx], dims[:nfx])) if nfx else 0
        col = int(np.ravel_multi_index(idx[nfx:], dims[nfx:])) if r > nfx else 0
        v = float(xm[row] @ ym[:, col]) * transpose_sign_at(legs, perm, idx)
        idx_out.append(tuple(idx[p] for p in perm))
        vals.append(v)
    return idx_out, np.array(vals)
