"""Pins of the oracle's lattice tables against the paper and the mathematics.

* velocity convention c_0 = (-1,0,0) = -c_10 (Section 2.6, beside the worked example)
* weights: quadrature identities of the D3Q19 / D3Q27 velocity sets (c_s^2 = 1/3, Section 2.6)
* the exact inverse moment matrix reproduces the worked example of Section 2.6
  (golden fixture tests/golden/worked_example_d3q19.txt)
* the equilibrium symmetry E_kbar = E_k - 6 rho t_k c_k.u (Section 2.6)
"""
import os

import numpy as np
import pytest

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("Q", [19, 27])
def test_velocity_set_structure(Q):
    c, t, opp = O.lattice(Q)
    assert len({tuple(v) for v in c}) == Q
    assert np.all(np.abs(c) <= 1)
    if Q == 19:
        assert np.all((c * c).sum(1) <= 2)
    h = (Q - 1) // 2
    assert np.all(c[h] == 0)
    for k in range(Q):
        assert np.all(c[opp[k]] == -c[k])
        if k < h:
            assert opp[k] == k + h + 1
            nz = c[k][np.nonzero(c[k])[0][0]]
            assert nz == -1  # first non-zero component is -1 in the first half


def test_paper_velocity_convention():
    c, _, opp = O.lattice(19)
    assert tuple(c[0]) == (-1, 0, 0)
    assert tuple(c[10]) == (1, 0, 0)
    assert opp[0] == 10


@pytest.mark.parametrize("Q", [19, 27])
def test_weight_quadrature(Q):
    """Isotropy up to fourth order with c_s^2 = 1/3: these identities fix the weights uniquely
    for the given velocity shells."""
    c, t, _ = O.lattice(Q)
    cs2 = 1.0 / 3.0
    assert abs(t.sum() - 1.0) < 1e-15
    for a in range(3):
        assert abs((t * c[:, a]).sum()) < 1e-16
        for b in range(3):
            assert abs((t * c[:, a] * c[:, b]).sum() - (cs2 if a == b else 0.0)) < 1e-15
            for g in range(3):
                assert abs((t * c[:, a] * c[:, b] * c[:, g]).sum()) < 1e-16
    assert abs((t * c[:, 0] ** 4).sum() - 3 * cs2 * cs2) < 1e-15
    assert abs((t * c[:, 0] ** 2 * c[:, 1] ** 2).sum() - cs2 * cs2) < 1e-15


def _golden_rows():
    rows = {}
    with open(os.path.join(HERE, "golden", "worked_example_d3q19.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, p, q, r, v = line.split()
            rows.setdefault(int(k), {})[(int(p), int(q), int(r))] = float(v)
    return rows


def test_worked_example_inverse():
    """Rows 0 and 10 of T^-1 are exactly the paper's f_0^out and f_10^out expressions."""
    pqr, Tinv = O.moment_basis(19)
    rows = _golden_rows()
    for k, coeffs in rows.items():
        for j in range(19):
            expect = coeffs.get(tuple(int(v) for v in pqr[j]), 0.0)
            assert Tinv[k, j] == expect, (k, tuple(pqr[j]), Tinv[k, j], expect)


def test_worked_example_difference():
    """f_0 = f_10 - rho (u_x - M*_120 - M*_102) (the difference equation of Section 2.6)."""
    pqr, Tinv = O.moment_basis(19)
    idx = {tuple(int(v) for v in p): j for j, p in enumerate(pqr)}
    d = Tinv[0] - Tinv[10]
    expect = np.zeros(19)
    expect[idx[(1, 0, 0)]] = -1.0
    expect[idx[(1, 2, 0)]] = 1.0
    expect[idx[(1, 0, 2)]] = 1.0
    assert np.array_equal(d, expect)


@pytest.mark.parametrize("Q", [19, 27])
def test_inverse_is_inverse(Q):
    c, _, _ = O.lattice(Q)
    pqr, Tinv = O.moment_basis(Q)
    T = np.array([[np.prod(c[k].astype(float) ** pqr[j]) for k in range(Q)] for j in range(Q)])
    assert np.abs(Tinv @ T - np.eye(Q)).max() < 1e-14
    assert np.abs(T @ Tinv - np.eye(Q)).max() < 1e-14


@pytest.mark.parametrize("Q", [19, 27])
def test_equilibrium_symmetry(Q):
    c, t, opp = O.lattice(Q)
    g = np.random.default_rng(5)
    for _ in range(20):
        rho = 1 + 0.1 * g.standard_normal()
        u = 0.05 * g.standard_normal(3)
        E = O.equilibrium(Q, 0, rho, u)
        for k in range(Q):
            assert abs(E[opp[k]] - (E[k] - 6 * rho * t[k] * (c[k] @ u))) < 1e-16


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("kind", [0, 1])
def test_equilibrium_moments(Q, kind):
    """Both equilibria carry density rho, momentum rho u and momentum flux rho(u u + c_s^2 I)."""
    c, t, _ = O.lattice(Q)
    rho, u = 1.07, np.array([0.03, -0.02, 0.01])
    E = O.equilibrium(Q, kind, rho, u)
    assert abs(E.sum() - rho) < 1e-15
    assert np.abs(c.T @ E - rho * u).max() < 1e-16
    P = np.einsum("k,ka,kb->ab", E, c, c)
    assert np.abs(P - rho * (np.outer(u, u) + np.eye(3) / 3)).max() < 1e-15
