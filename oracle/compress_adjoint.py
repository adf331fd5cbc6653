"""Adjoint (gradient) of the sector-wise QR/SVD bond compression of
:func:`oracle.compress.compress` (Sec. II.A, Sec. II.B).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Per bond-parity sector the compression computes X_pi = Q_X R_X and
Y_pi^T = Q_Y R_Y (thin QR), the core M = R_X R_Y^T = U S V^T (thin SVD), keeps
the k largest singular values of all sectors, and returns X' = Q_X U_k S_k^1/2
and Y' = S_k^1/2 V_k^T Q_Y^T.  For a scalar L(X', Y') with cotangents
G_X' = dL/dX' and G_Y' = dL/dY', the gradient with respect to X and Y is
obtained by running these steps backwards, each with its reverse-mode rule:

* the products and the column scaling by S_k^1/2: the chain rule;
* the thin SVD M = U S V^T (J. Townsend, "Differentiating the singular value
  decomposition", 2016):
      dM = U [ (F o (U^T dU - dU^T U)) S + diag(dS) + S (F o (V^T dV - dV^T V)) ] V^T
           + (I - U U^T) dU S^-1 V^T + U S^-1 dV^T (I - V V^T),
  F_ij = 1 / (s_j^2 - s_i^2) for i != j and 0 on the diagonal.  Only the kept
  columns carry cotangents, so a pair of discarded columns contributes nothing
  and its F entry (possibly 1/0 for repeated discarded values) is not formed;
* the thin QR A = Q R (S. F. Walter and L. Lehmann, "Algorithmic
  differentiation of linear algebra functions with application in optimum
  experimental design", 2013; in the form of H.-J. Liao et al.,
  "Differentiable programming tensor networks", 2019): for m >= n,
      dA = [dQ + Q copyltu(R dR^T - dQ^T Q)] R^-T,
      copyltu(B) = tril(B) + tril(B, -1)^T;
  for m < n, A = Q [R1 | R2] with R1 square (Q is the QR factor of the left
  block A1 and R2 = Q^T A2): dA2 = Q dR2, and the square rule gives dA1 from
  dQ + A2 dR2^T and dR1;
* the matricisation (fermionic transposes and bond-parity flips, linear with
  +-1 signs): by its definition, one parity-allowed entry at a time, as in
  :mod:`oracle.adjoint`.

The rules hold where the compression is differentiable: a gap at the
truncation cut (the kept set does not change), singular values distinct among
and against the kept ones, and full-rank sector blocks (invertible R).  The
forward factors are recomputed here with the same numpy calls as
:func:`oracle.compress.compress` (checked equal to its output by the tests).
"""
from __future__ import annotations

import itertools

import numpy as np

from .compress import matricize_pair
from .graded import GTensor, index_parity

__all__ = ["compress_factors", "compress_grad"]


def _svd_backward(u, s, v, du, ds, dv, keep):
    """dL/dM for M = u diag(s) v^T (thin), given the cotangents of u, s, v;
    only the first ``keep`` columns of du and dv may be nonzero."""
    r = len(s)
    f = np.zeros((r, r))
    for i in range(r):
        for j in range(r):
            if i != j and (i < keep or j < keep):
                f[i, j] = 1.0 / (s[j] ** 2 - s[i] ** 2)
    jm = f * (u.T @ du - du.T @ u)
    km = f * (v.T @ dv - dv.T @ v)
    sm = np.diag(s)
    dm = u @ (jm @ sm + np.diag(ds) + sm @ km) @ v.T
    sinv = np.zeros(r)
    sinv[:keep] = 1.0 / s[:keep]
    dm = dm + (np.eye(u.shape[0]) - u @ u.T) @ du @ np.diag(sinv) @ v.T
    dm = dm + u @ np.diag(sinv) @ dv.T @ (np.eye(v.shape[0]) - v @ v.T)
    return dm


def _copyltu(b):
    return np.tril(b) + np.tril(b, -1).T


def _qr_backward(a, q, r, dq, dr):
    """dL/dA for the thin QR A = q r, given the cotangents of q and r."""
    m, n = a.shape
    if m >= n:
        c = _copyltu(r @ dr.T - dq.T @ q)
        # (dq + q c) R^-T: solve R X^T = (dq + q c)^T
        return np.linalg.solve(r, (dq + q @ c).T).T
    a2 = a[:, m:]
    dr1, dr2 = dr[:, :m], dr[:, m:]
    da1 = _qr_backward(a[:, :m], q, r[:, :m], dq + a2 @ dr2.T, dr1)
    return np.concatenate([da1, q @ dr2], axis=1)


def compress_factors(x, y, ax, ay, chi, arrows=True):
    """The forward steps of :func:`oracle.compress.compress`, keeping the
    factors: returns (xm, ym, sectors, kept) with sectors[pi] = (rows, ks,
    cols, (qx, rx, qy, ry, u, s, vt) or None) and kept = (k0, k1)."""
    xm, ym, fx, fy, rpar, kpar, cpar = matricize_pair(x, y, ax, ay, arrows=arrows)
    px, py = x.parity, y.parity
    sec = {}
    cand = []
    for pi in (0, 1):
        rows = np.nonzero(rpar == (px ^ pi))[0]
        ks = np.nonzero(kpar == pi)[0]
        cols = np.nonzero(cpar == (py ^ pi))[0]
        fac = None
        if len(rows) and len(ks) and len(cols):
            xp = xm[np.ix_(rows, ks)]
            yp = ym[np.ix_(ks, cols)]
            qx, rx = np.linalg.qr(xp)
            qy, ry = np.linalg.qr(yp.T)
            u, s, vt = np.linalg.svd(rx @ ry.T, full_matrices=False)
            fac = (qx, rx, qy, ry, u, s, vt)
            for i, sv in enumerate(s):
                cand.append((-float(sv), pi, i))
        sec[pi] = (rows, ks, cols, fac)
    cand.sort()
    kept = cand[: max(int(chi), 0)]
    k = tuple(sum(1 for c in kept if c[1] == pi) for pi in (0, 1))
    return xm, ym, sec, k


def _allowed(t):
    par = [index_parity(d0, d1) for d0, d1, _ in t.legs]
    for idx in itertools.product(*[range(len(p)) for p in par]):
        if sum(int(par[k][i]) for k, i in enumerate(idx)) % 2 == t.parity:
            yield idx


def compress_grad(x, y, ax, ay, chi, gx, gy, arrows=True):
    """(dL/dX, dL/dY) as GTensors for a scalar L(X', Y') with cotangents
    gx = dL/dX' and gy = dL/dY' (GTensors with the legs of the X' and Y' that
    ``compress(x, y, ax, ay, chi, arrows)`` returns)."""
    xm, ym, sec, k = compress_factors(x, y, ax, ay, chi, arrows)
    nk = k[0] + k[1]
    gxm = gx.data.reshape(xm.shape[0], nk)
    gym = gy.data.reshape(nk, ym.shape[1])
    dxm = np.zeros(xm.shape)
    dym = np.zeros(ym.shape)
    off = {0: 0, 1: k[0]}
    for pi in (0, 1):
        rows, ks, cols, fac = sec[pi]
        kk = k[pi]
        if fac is None or kk == 0:
            continue
        qx, rx, qy, ry, u, s, vt = fac
        v = vt.T
        new = np.arange(off[pi], off[pi] + kk)
        g_x = gxm[np.ix_(rows, new)]        # dL/dX' of this sector (m x kk)
        g_yt = gym[np.ix_(new, cols)].T     # dL/d(Y'^T) of this sector (n x kk)
        rs = np.sqrt(s[:kk])
        ut = u[:, :kk] * rs                 # X' = qx ut
        vtl = v[:, :kk] * rs                # Y'^T = qy vtl
        dqx = g_x @ ut.T
        dut = qx.T @ g_x
        dqy = g_yt @ vtl.T
        dvt = qy.T @ g_yt
        du = np.zeros(u.shape)
        dv = np.zeros(v.shape)
        du[:, :kk] = dut * rs
        dv[:, :kk] = dvt * rs
        ds = np.zeros(len(s))
        ds[:kk] = (np.sum(dut * u[:, :kk], axis=0) + np.sum(dvt * v[:, :kk], axis=0)) / (2.0 * rs)
        dm = _svd_backward(u, s, v, du, ds, dv, kk)
        drx = dm @ ry                       # M = rx ry^T
        dry = dm.T @ rx
        xp = xm[np.ix_(rows, ks)]
        ypt = ym[np.ix_(ks, cols)].T
        dxm[np.ix_(rows, ks)] += _qr_backward(xp, qx, rx, dqx, drx)
        dym[np.ix_(ks, cols)] += _qr_backward(ypt, qy, ry, dqy, dry).T
    # the matricisation is linear in each operand: its adjoint entry by entry
    dx = np.zeros(x.data.shape)
    for idx in _allowed(x):
        e = np.zeros(x.data.shape)
        e[idx] = 1.0
        em = matricize_pair(GTensor(e, x.legs, x.parity), y, ax, ay, arrows=arrows)[0]
        dx[idx] = float(np.sum(dxm * em))
    dy = np.zeros(y.data.shape)
    for idx in _allowed(y):
        e = np.zeros(y.data.shape)
        e[idx] = 1.0
        em = matricize_pair(x, GTensor(e, y.legs, y.parity), ax, ay, arrows=arrows)[1]
        dy[idx] = float(np.sum(dym * em))
    return GTensor(dx, x.legs, x.parity), GTensor(dy, y.legs, y.parity)
