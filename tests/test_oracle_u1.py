"""Pins of the U(1) x parity structure (oracle.u1): fermion-number charges
whose parity is the charge mod 2 (Sec. II.B).

* the Z2 leg of a U(1) leg and the parity of a charged tensor follow the
  charges (even charges even);
* the Hubbard hopping and on-site gates conserve the fermion number (Q = 0
  with charges 0, 2, 1, 1 on the physical leg);
* a contraction of U(1)-symmetric tensors, by the Z2 oracle, is
  U(1)-symmetric with total charge Q_X + Q_Y (exactly: every product outside
  the allowed set has a zero factor);
* the compression of a U(1)-symmetric pair keeps the symmetry: every state
  of the new bond has one definite charge (to rounding), and op(X', Y')
  stays within the allowed set of op(X, Y).
"""
import numpy as np
import pytest

import oracle as O
import oracle.u1 as U

CASES = [
    # U(1) legs of X and Y, contracted axes, total charges
    ([([(0, 1), (1, 2), (-1, 1)], 0), ([(0, 2), (1, 1), (2, 1)], 1), ([(1, 1), (0, 1), (2, 1)], 0)],
     [([(1, 1), (0, 1), (2, 1)], 1), ([(0, 1), (1, 1), (-1, 2)], 0)], [2], [0], 1, 0),
    ([(U.HUBBARD_SITE, 0), ([(0, 2), (1, 2), (-1, 1)], 1), ([(0, 1), (2, 2), (1, 1)], 0)],
     [([(0, 2), (1, 2), (-1, 1)], 0), ([(1, 2), (0, 1)], 1), ([(0, 1), (2, 2), (1, 1)], 1)], [1, 2], [0, 2], 2, -1),
]


def test_z2_legs_and_parity_follow_the_charges():
    leg, q = U.u1_leg([(1, 2), (0, 1), (2, 3), (-1, 1)], 1)
    assert leg == (4, 3, 1)
    assert list(q) == [0, 2, 2, 2, 1, 1, -1]
    t = U.random_u1([([(0, 1), (1, 1)], 0), ([(0, 1), (1, 1)], 0)], 1, 3)
    assert t.parity == 1 and t.check_symmetry()


def test_hubbard_gates_conserve_fermion_number():
    legs = [(U.HUBBARD_SITE, 0), (U.HUBBARD_SITE, 0), (U.HUBBARD_SITE, 1), (U.HUBBARD_SITE, 1)]
    assert U.u1_z2_legs(legs) == [(2, 2, 0)] * 2 + [(2, 2, 1)] * 2
    hop = O.hop_gate(1.0)
    assert np.max(np.abs(hop.data)) > 0 and U.u1_violation(hop, legs, 0) == 0.0
    site = O.onsite_gate(8.0)
    assert U.u1_violation(site, [(U.HUBBARD_SITE, 0), (U.HUBBARD_SITE, 1)], 0) == 0.0
    # a gate moving one fermion is not number-conserving: the check sees it
    bad = O.GTensor(np.roll(hop.data, 1, axis=0), hop.legs, hop.parity)
    assert U.u1_violation(bad, legs, 0) > 0


@pytest.mark.parametrize("case", CASES)
def test_contraction_conserves_the_charge(case):
    lx, ly, ax, ay, qx, qy = case
    x, y = U.random_u1(lx, qx, 1), U.random_u1(ly, qy, 2)
    assert U.u1_violation(x, lx, qx) == 0.0 and U.u1_violation(y, ly, qy) == 0.0
    z = O.contract(x, y, ax, ay)
    lz = U.u1_result_legs(lx, ly, ax, ay)
    assert np.max(np.abs(z.data)) > 0
    assert U.u1_violation(z, lz, qx + qy) == 0.0
    assert z.parity == (qx + qy) % 2


@pytest.mark.parametrize("case", CASES)
def test_compression_keeps_the_symmetry(case):
    lx, ly, ax, ay, qx, qy = case
    x, y = U.random_u1(lx, qx, 3), U.random_u1(ly, qy, 4)
    _, _, info = O.compress(x, y, ax, ay, chi=10**6)
    chi = max(1, len(info["singular_values"]) // 2)
    xn, yn, _ = O.compress(x, y, ax, ay, chi)
    # every new bond state (a column of X' over X's free indices) has one charge
    fx = [lx[k] for k in range(len(lx)) if k not in ax]
    free_charge = np.zeros([1] * len(fx), np.int64)
    for k, (s, du) in enumerate(fx):
        _, q = U.u1_leg(s, du)
        shp = [1] * len(fx)
        shp[k] = len(q)
        free_charge = free_charge + (1 if du == 0 else -1) * q.reshape(shp)
    free_charge = np.broadcast_to(free_charge, xn.data.shape[:-1]).reshape(-1)
    xm = xn.data.reshape(-1, xn.data.shape[-1])
    scale = np.max(np.abs(xm))
    for c in range(xm.shape[1]):
        col = xm[:, c]
        big = np.abs(col) > 1e-10 * scale
        assert big.any() and len(set(free_charge[big])) == 1
    z = O.contract(xn, yn, [xn.rank - 1], [0])
    lz = U.u1_result_legs(lx, ly, ax, ay)
    assert U.u1_violation(z, lz, qx + qy) <= 1e-12 * np.max(np.abs(z.data))
