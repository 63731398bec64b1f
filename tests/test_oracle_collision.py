"""Pins of the oracle's collision models, cell by cell.

Properties every model must have (Sections 2.1, 2.2, 2.6 of the paper):
conservation of mass and momentum, preservation of its own equilibrium, full
relaxation to equilibrium at omega = 1, the reduction of the linear moment
models to BGK-NW4 when all rates are equal, the per-moment relaxation law of
Section 2.6 (checked with moments computed here, independently of the oracle's
transforms), the bulk-viscosity coupling, and the cumulant definition checked
against derivatives of the log moment-generating function.
"""
import numpy as np
import pytest
import sympy as sp

from oracle import oracle as O

MODELS = list(O.MODELS)
CS2 = 1.0 / 3.0


def _rand_f(Q, seed, amp=0.3):
    _, t, _ = O.lattice(Q)
    g = np.random.default_rng(seed)
    return t * (1.0 + amp * g.uniform(-1, 1, Q)) * (1.0 + 0.05 * g.standard_normal())


def _rho_u(Q, f):
    c, _, _ = O.lattice(Q)
    rho = f.sum()
    return rho, (c.T @ f) / rho


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("model", MODELS)
def test_conservation(Q, model):
    c, _, _ = O.lattice(Q)
    for s in range(10):
        f = _rand_f(Q, s)
        prm = O.params(1.2 + 0.07 * s, 0.9 + 0.05 * s, 1.1, 0.2)
        fo = O.collide(Q, model, prm, f)
        assert abs(fo.sum() - f.sum()) <= 1e-13 * f.sum()
        assert np.abs(c.T @ fo - c.T @ f).max() <= 1e-13 * f.sum()


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("model", MODELS)
def test_equilibrium_is_fixed_point(Q, model):
    for s in range(5):
        g = np.random.default_rng(100 + s)
        rho, u = 1 + 0.05 * g.standard_normal(), 0.04 * g.standard_normal(3)
        E = O.model_equilibrium(Q, model, rho, u)
        fo = O.collide(Q, model, O.params(1.6, 1.1, 0.8, 0.3), E)
        assert np.abs(fo - E).max() < 1e-15


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("model", MODELS)
def test_omega_one_gives_equilibrium(Q, model):
    for s in range(5):
        f = _rand_f(Q, 200 + s)
        rho, u = _rho_u(Q, f)
        fo = O.collide(Q, model, O.params(1.0, 1.0, 1.0, 0.25), f)
        assert np.abs(fo - O.model_equilibrium(Q, model, rho, u)).max() < 2e-16


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("model", ["RM", "HM", "CM", "CHM"])
def test_equal_rates_reduce_to_bgk_nw4(Q, model):
    for s in range(5):
        f = _rand_f(Q, 300 + s)
        w = 0.7 + 0.2 * s
        ref = O.collide(Q, "BGK_NW4", O.params(w), f)
        got = O.collide(Q, model, O.params(w, w, w), f)
        assert np.abs(got - ref).max() < 5e-16


def _moment_matrix(Q, shift=(0.0, 0.0, 0.0), hermite=False):
    """Rows: basis polynomials evaluated at c_k - shift (monomial or Hermite)."""
    c, _, _ = O.lattice(Q)
    pqr, _ = O.moment_basis(Q)
    xi = c.astype(float) - np.asarray(shift)[None, :]

    def p1(p, v):
        if p == 0:
            return np.ones_like(v)
        if p == 1:
            return v
        return v * v - (CS2 if hermite else 0.0)

    return np.array([p1(a, xi[:, 0]) * p1(b, xi[:, 1]) * p1(g, xi[:, 2]) for a, b, g in pqr]), pqr


def _check_relaxation(Q, X, Xs, Xeq, pqr, w, wb, wh, skip_high=False):
    order = pqr.sum(1)
    d = [int(np.where((pqr == e).all(1))[0][0]) for e in ([2, 0, 0], [0, 2, 0], [0, 0, 2])]
    wm = (wb - w) / 3.0
    wp = wm + w
    for j in range(Q):
        if order[j] == 2 and j not in d:
            assert abs(Xs[j] - (X[j] - w * (X[j] - Xeq[j]))) < 1e-15
        elif order[j] >= 3 and not skip_high:
            assert abs(Xs[j] - (X[j] - wh * (X[j] - Xeq[j]))) < 1e-15
    for a in range(3):
        expect = X[d[a]] - sum((wp if b == a else wm) * (X[d[b]] - Xeq[d[b]]) for b in range(3))
        assert abs(Xs[d[a]] - expect) < 1e-15
    # trace relaxes with the bulk rate, the deviatoric part with omega
    tr = sum(X[i] - Xeq[i] for i in d)
    trs = sum(Xs[i] - Xeq[i] for i in d)
    assert abs(trs - (1 - wb) * tr) < 1e-15
    dev = (X[d[0]] - Xeq[d[0]]) - (X[d[1]] - Xeq[d[1]])
    devs = (Xs[d[0]] - Xeq[d[0]]) - (Xs[d[1]] - Xeq[d[1]])
    assert abs(devs - (1 - w) * dev) < 1e-15


def _m1(p, u):
    return 1.0 if p == 0 else (u if p == 1 else u * u + CS2)


@pytest.mark.parametrize("Q", [19, 27])
def test_raw_moment_relaxation_law(Q):
    w, wb, wh = 1.7, 1.2, 0.9
    for s in range(4):
        f = _rand_f(Q, 400 + s)
        rho, u = _rho_u(Q, f)
        fo = O.collide(Q, "RM", O.params(w, wb, wh), f)
        T, pqr = _moment_matrix(Q)
        X, Xs = T @ f / rho, T @ fo / rho
        Xeq = np.array([_m1(a, u[0]) * _m1(b, u[1]) * _m1(g, u[2]) for a, b, g in pqr])
        _check_relaxation(Q, X, Xs, Xeq, pqr, w, wb, wh)


@pytest.mark.parametrize("Q", [19, 27])
def test_hermite_moment_relaxation_law(Q):
    w, wb, wh = 1.6, 0.8, 1.3
    for s in range(4):
        f = _rand_f(Q, 500 + s)
        rho, u = _rho_u(Q, f)
        fo = O.collide(Q, "HM", O.params(w, wb, wh), f)
        T, pqr = _moment_matrix(Q, hermite=True)
        X, Xs = T @ f / rho, T @ fo / rho
        Xeq = np.array([u[0] ** a * u[1] ** b * u[2] ** g for a, b, g in pqr])
        _check_relaxation(Q, X, Xs, Xeq, pqr, w, wb, wh)


@pytest.mark.parametrize("Q", [19, 27])
@pytest.mark.parametrize("model,hermite", [("CM", False), ("CHM", True)])
def test_central_moment_relaxation_law(Q, model, hermite):
    w, wb, wh = 1.5, 1.0, 1.2
    for s in range(4):
        f = _rand_f(Q, 600 + s)
        rho, u = _rho_u(Q, f)
        fo = O.collide(Q, model, O.params(w, wb, wh), f)
        T, pqr = _moment_matrix(Q, shift=u, hermite=hermite)  # collision conserves u
        X, Xs = T @ f / rho, T @ fo / rho
        if hermite:
            Xeq = np.array([1.0 if (a, b, g) == (0, 0, 0) else 0.0 for a, b, g in pqr])
        else:
            Xeq = np.array([_m1(a, 0.0) * _m1(b, 0.0) * _m1(g, 0.0) for a, b, g in pqr])
        _check_relaxation(Q, X, Xs, Xeq, pqr, w, wb, wh)


@pytest.mark.parametrize("Q", [19, 27])
def test_trt_parts(Q):
    """TRT: the symmetric non-equilibrium part relaxes with omega, the antisymmetric with
    omega_minus fixed by Lambda = (1/w+ - 1/2)(1/w- - 1/2)."""
    _, _, opp = O.lattice(Q)
    w, lam = 1.7, 0.3
    wm = 1.0 / (0.5 + lam / (1.0 / w - 0.5))
    for s in range(4):
        f = _rand_f(Q, 700 + s)
        rho, u = _rho_u(Q, f)
        E = O.equilibrium(Q, 0, rho, u)
        fo = O.collide(Q, "TRT", O.params(w, trt_lambda=lam), f)
        n, no = f - E, fo - E
        sym, asym = 0.5 * (n + n[opp]), 0.5 * (n - n[opp])
        assert np.abs(0.5 * (no + no[opp]) - (1 - w) * sym).max() < 1e-16
        assert np.abs(0.5 * (no - no[opp]) - (1 - wm) * asym).max() < 1e-16


@pytest.mark.parametrize("Q", [19, 27])
def test_regularized_projection(Q):
    """REG: the post-collision non-equilibrium is t_k H2_k : A for a symmetric A, and its
    momentum flux is (1 - omega) times the incoming non-equilibrium flux."""
    c, t, _ = O.lattice(Q)
    w = 1.4
    for s in range(4):
        f = _rand_f(Q, 800 + s)
        rho, u = _rho_u(Q, f)
        E = O.equilibrium(Q, 0, rho, u)
        fo = O.collide(Q, "REG", O.params(w), f)
        Pi_in = np.einsum("k,ka,kb->ab", f - E, c, c)
        Pi_out = np.einsum("k,ka,kb->ab", fo - E, c, c)
        assert np.abs(Pi_out - (1 - w) * Pi_in).max() < 1e-15
        H = np.array([[c[k, a] * c[k, b] - (CS2 if a == b else 0) for a in range(3) for b in range(3)]
                      for k in range(Q)]) * t[:, None]
        coef, *_ = np.linalg.lstsq(H, fo - E, rcond=None)
        assert np.abs(H @ coef - (fo - E)).max() < 1e-15


def test_rr_equals_reg_at_rest_d3q27():
    """At zero velocity the recursive high-order terms vanish; on D3Q27 (Hermite-orthogonal
    up to the basis) RR then coincides with the plain regularized model."""
    c, t, opp = O.lattice(27)
    for s in range(4):
        f = _rand_f(27, 900 + s)
        f = 0.5 * (f + f[opp])  # symmetric part only: zero momentum
        rr = O.collide(27, "RR", O.params(1.3), f)
        reg = O.collide(27, "REG", O.params(1.3), f)
        assert np.abs(rr - reg).max() < 1e-15


def _mgf_cumulant(Q, f, e):
    """Brute force: d^n/d(lambda) log sum_k f_k exp(lambda.(c_k - u)) at 0, exact rationals."""
    c, _, _ = O.lattice(Q)
    lx, ly, lz = sp.symbols("lx ly lz")
    fr = [sp.Rational(int(round(v * 2 ** 20)), 2 ** 20) for v in f]
    rho = sum(fr)
    u = [sum(fr[k] * int(c[k, d]) for k in range(Q)) / rho for d in range(3)]
    mgf = sum(fr[k] * sp.exp(lx * (int(c[k, 0]) - u[0]) + ly * (int(c[k, 1]) - u[1]) + lz * (int(c[k, 2]) - u[2]))
              for k in range(Q)) / rho
    expr = sp.log(mgf)
    for sym, n in zip((lx, ly, lz), e):
        if n:
            expr = sp.diff(expr, sym, n)
    return float(expr.subs({lx: 0, ly: 0, lz: 0})), np.array([float(v) for v in fr])


@pytest.mark.parametrize("Q,elems", [(19, [(1, 1, 0), (1, 2, 0), (2, 2, 0), (0, 2, 2)]),
                                     (27, [(2, 2, 0), (2, 1, 1), (2, 2, 1), (2, 2, 2)])])
def test_cumulants_match_log_mgf(Q, elems):
    pqr, _ = O.moment_basis(Q)
    f0 = _rand_f(Q, 1000, amp=0.5)
    for e in elems:
        ref, fq = _mgf_cumulant(Q, f0, e)
        K = O.cumulants(Q, fq)
        j = int(np.where((pqr == np.array(e)).all(1))[0][0])
        assert abs(K[j] - ref) < 1e-14 * max(1.0, abs(ref)), (e, K[j], ref)


def test_cumulants_of_product_distribution_d3q27():
    """A product of three 1-D distributions has vanishing mixed cumulants and per-axis variances."""
    c, _, _ = O.lattice(27)
    pqr, _ = O.moment_basis(27)
    g = np.random.default_rng(11)
    p1d = [g.uniform(0.2, 1.0, 3) for _ in range(3)]
    p1d = [p / p.sum() for p in p1d]
    f = np.array([1.3 * p1d[0][c[k, 0] + 1] * p1d[1][c[k, 1] + 1] * p1d[2][c[k, 2] + 1] for k in range(27)])
    K = O.cumulants(27, f)
    for j, e in enumerate(pqr):
        if (e > 0).sum() >= 2:
            assert abs(K[j]) < 1e-15, tuple(e)
    v = np.array([-1.0, 0.0, 1.0])
    for a in range(3):
        mean = (p1d[a] * v).sum()
        var = (p1d[a] * (v - mean) ** 2).sum()
        j = int(np.where((pqr == np.eye(3, dtype=int)[a] * 2).all(1))[0][0])
        assert abs(K[j] - var) < 1e-15


@pytest.mark.parametrize("Q", [19, 27])
def test_cumulant_relaxation_law(Q):
    """K: post-collision cumulants follow the relaxation law (second order towards c_s^2 delta,
    higher orders towards 0 with omega_high)."""
    pqr, _ = O.moment_basis(Q)
    w, wb, wh = 1.3, 1.0, 0.7
    for s in range(3):
        f = _rand_f(Q, 1100 + s)
        fo = O.collide(Q, "K", O.params(w, wb, wh), f)
        K, Ks = O.cumulants(Q, f), O.cumulants(Q, fo)
        Keq = np.array([CS2 if (sorted(e) == [0, 0, 2]) else 0.0 for e in pqr])
        _check_relaxation(Q, K, Ks, Keq, pqr, w, wb, wh)


def _rr_expected_high(pqr, u, n2):
    """Order >= 3 Hermite moments the recursive regularization prescribes, by a route of
    its own: each is m(u) + 1/2 sum_ab n2_ab d^2 m / du_a du_b with m(u) = ux^p uy^q uz^r.
    The second derivative picks every unordered pair of the moment's index multiset once
    (p_a p_b pairs for a != b, p_a (p_a - 1)/2 for a = b), so this is the sum over index
    pairs of n2_pair times the product of the remaining velocities, with the pair counts
    supplied by calculus rather than by an enumeration of indices."""
    us = sp.symbols("ux uy uz")
    sub = dict(zip(us, [float(v) for v in u]))
    out = {}
    for j, (p, q, r) in enumerate(pqr):
        if p + q + r < 3:
            continue
        m = us[0] ** int(p) * us[1] ** int(q) * us[2] ** int(r)
        corr = sum(sp.Rational(1, 2) * n2[a][b] * sp.diff(m, us[a], us[b]) for a in range(3) for b in range(3))
        out[j] = float((m + corr).subs(sub))
    return out


@pytest.mark.parametrize("Q", [19, 27])
def test_rr_recursive_high_order_moments(Q):
    """RR (recursive regularization, Section 2.2 list of models; moment route of Section 2.6):
    at u ~ 0.1 and omega != 1, with the bulk coupling on and omega_high != 1 (which RR
    ignores), the post-collision Hermite moments computed here from f_out satisfy
      * second order: the relaxation law with the bulk coupling;
      * order >= 3: X*_j = prod u + sum over index pairs of neq2*_pair prod(remaining u),
        where neq2* = X*_2 - prod u is the post-collision second-order non-equilibrium.
    A dropped pair, a swapped axis or a u written for a neq2 term moves an order-3 moment
    by ~1e-3 and an order-6 one by ~1e-7, both far above the 1e-15 tolerance."""
    c, t, _ = O.lattice(Q)
    T, pqr = _moment_matrix(Q, hermite=True)
    w, wb, wh = 1.6, 1.1, 0.7
    for s in range(4):
        g = np.random.default_rng(1200 + s)
        u0 = np.array([0.11, -0.08, 0.06]) * (1.0 + 0.3 * g.uniform(-1, 1, 3))
        f = O.equilibrium(Q, 0, 1.0 + 0.05 * g.standard_normal(), u0) * (1.0 + 0.04 * g.standard_normal(Q))
        rho, u = _rho_u(Q, f)
        assert np.abs(u).min() > 0.03  # the recursive terms are not negligible here
        fo = O.collide(Q, "RR", O.params(w, wb, wh), f)
        X, Xs = T @ f / rho, T @ fo / rho
        Xeq = np.array([u[0] ** a * u[1] ** b * u[2] ** gg for a, b, gg in pqr])
        _check_relaxation(Q, X, Xs, Xeq, pqr, w, wb, wh, skip_high=True)
        n2 = [[0.0] * 3 for _ in range(3)]
        for a in range(3):
            for b in range(3):
                e = [0, 0, 0]
                e[a] += 1
                e[b] += 1
                j = int(np.where((pqr == np.array(e)).all(1))[0][0])
                n2[a][b] = Xs[j] - Xeq[j]
        want = _rr_expected_high(pqr, u, n2)
        assert len(want) == (9 if Q == 19 else 17)  # D3Q19: 6 of order 3, 3 of order 4
        for j, v in want.items():
            assert abs(Xs[j] - v) < 1e-15, (tuple(pqr[j]), Xs[j], v)
            # the recursive part is exercised far above the tolerance (order 3: ~1e-3)
            assert abs(v - Xeq[j]) > 1e-9
