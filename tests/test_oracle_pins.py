"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test reaches the expected value by a route that does not go through the
oracle's own arithmetic: printed constants of the paper, textbook quadrature
weights, a symbolic derivation from the continuous stage equation
(eq. MB4_1), brute-force quadrature and root finding, a library ODE solver,
and invariants (energy, translation, time reversal, plane waves).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.integrate
import scipy.interpolate
import scipy.optimize

from oracle import mb4_oracle as orc
from paper_2003_04345_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            out[parts[0]] = parts[1:]
    return out


PAPER = _golden("paper_constants.txt")
TEXTBOOK = _golden("textbook_values.txt")
ALPHA_PAPER = Fraction(int(PAPER["alpha1_paper_num"][0]), int(PAPER["alpha1_paper_den"][0]))
C_PAPER = tuple(Fraction(PAPER[k][0]) for k in ("c1", "c2", "c3"))


# ---------------------------------------------------------------------------
# Independent brute-force stage residual: numerical quadrature of eq. (MB4_3)
# with a 20-point Gauss-Legendre rule (exact to degree 39), the stage
# polynomial from scipy's Lagrange interpolation, A from eq. (Adefinition) in
# floats, and f from np.roll stencils.  No E matrix, no cubic tensor.
# ---------------------------------------------------------------------------
def _A_float(alpha, tau, zeta):
    a = float(alpha)
    M = np.array([[a + 4, -6 * a - 6, 6 * a],
                  [-6 * a - 6, 36 * a + 12, -36 * a],
                  [6 * a, -36 * a, 36 * a]])
    return np.array([tau, tau ** 2 / 2, tau ** 3 / 3]) @ M @ np.array([1.0, zeta, zeta ** 2])


def _f_roll(u, nx, ny, V, chi, tx, ty, eps0):
    g = u.reshape(ny, nx)
    Ku = (eps0 * g - tx * (np.roll(g, 1, axis=1) + np.roll(g, -1, axis=1))
          - ty * (np.roll(g, 1, axis=0) + np.roll(g, -1, axis=0)))
    Ku = Ku.reshape(nx * ny)
    return -1j * (Ku + V * u + chi * np.abs(u) ** 2 * u)


def brute_phi(nx, ny, V, chi, tx, ty, eps0, u0, U, h, alpha=ALPHA_PAPER, c=C_PAPER, nq=20):
    nodes = np.array([0.0] + [float(x) for x in c])
    zq, wq = np.polynomial.legendre.leggauss(nq)
    zq = 0.5 * (zq + 1.0)
    wq = 0.5 * wq
    lag = scipy.interpolate.BarycentricInterpolator(nodes, np.eye(4))
    X = np.vstack([u0[None, :], U])
    acc = np.zeros_like(U)
    for z, w in zip(zq, wq):
        lz = lag(z)
        Uz = sum(lz[j] * X[j] for j in range(4))
        fz = _f_roll(Uz, nx, ny, V, chi, tx, ty, eps0)
        for i in range(3):
            acc[i] += w * _A_float(alpha, float(c[i]), z) * fz
    return U - u0[None, :] - h * acc


def _rand_state(rng, S, scale=1.0):
    return scale * (rng.normal(size=S) + 1j * rng.normal(size=S))


# ---------------------------------------------------------------------------
# Constants.
# ---------------------------------------------------------------------------
def test_last_row_of_E_is_simpson_three_eighths():
    """B_zeta = A_{1,zeta}, and with c3 = 1 the row E_3j = int B l_j is the
    4-node Newton-Cotes (Simpson 3/8) weight set."""
    k = orc.mb4_constants(ALPHA_PAPER, C_PAPER)
    want = [Fraction(x) for x in TEXTBOOK["simpson38"]]
    assert k["E"][2] == want


def test_E_row_sums_are_the_nodes():
    """Runge-Kutta row-sum condition: sum_{j=0..3} E_ij = c_i."""
    for c in (C_PAPER, (Fraction(1, 4), Fraction(1, 2), Fraction(1)), (Fraction(3, 10), Fraction(7, 10), Fraction(1))):
        k = orc.mb4_constants(ALPHA_PAPER, c)
        for i in range(3):
            assert sum(k["E"][i]) == c[i]


def test_E_eigenvalues_real_and_independent_of_nodes():
    """Sec. 2.2 (citing Miyatake-Butcher Thm 5.1): E is diagonalisable with real
    eigenvalues that do not depend on c1, c2, c3."""
    ev = []
    for c in (C_PAPER, (Fraction(1, 4), Fraction(1, 2), Fraction(1)), (Fraction(1, 5), Fraction(3, 5), Fraction(1))):
        E, _ = orc.constants_f64(ALPHA_PAPER, c)
        lam = np.linalg.eigvals(E[:, 1:])
        assert np.max(np.abs(lam.imag)) < 1e-12
        ev.append(np.sort(lam.real))
    for e in ev[1:]:
        assert np.allclose(e, ev[0], rtol=0, atol=1e-12)
    # The trace of E(1:3,1:3) equals the sum of the eigenvalues: a consistency check on the
    # numerical eigen-solve only.
    assert abs(sum(ev[0]) - np.trace(orc.constants_f64(ALPHA_PAPER, C_PAPER)[0][:, 1:])) < 1e-12


def _charpoly_disc(alpha):
    """Discriminant of det(x I - E(alpha)), exact (E from the oracle, Fractions)."""
    E = [row[1:] for row in orc.mb4_constants(Fraction(alpha), C_PAPER)["E"]]
    tr = E[0][0] + E[1][1] + E[2][2]
    m2 = (E[0][0] * E[1][1] - E[0][1] * E[1][0] + E[0][0] * E[2][2] - E[0][2] * E[2][0]
          + E[1][1] * E[2][2] - E[1][2] * E[2][1])
    det = (E[0][0] * (E[1][1] * E[2][2] - E[1][2] * E[2][1])
           - E[0][1] * (E[1][0] * E[2][2] - E[1][2] * E[2][0])
           + E[0][2] * (E[1][0] * E[2][1] - E[1][1] * E[2][0]))
    a, b, cc = -tr, m2, -det      # x^3 + a x^2 + b x + cc
    return 18 * a * b * cc - 4 * a ** 3 * cc + a * a * b * b - 4 * b ** 3 - 27 * cc * cc


def test_alpha1_bound_printed_in_paper():
    """The paper requires alpha1 < -300 * 0.7770503941 (Sec. 2.2).  The oracle's
    E(alpha) must switch from three real eigenvalues to a complex pair exactly
    there (to the 10 printed digits)."""
    factor = Fraction(PAPER["alpha1_bound_factor"][0])
    ab = -300 * factor
    eps = Fraction(300 * 6, 10 ** 11)          # half a unit in the last printed digit, x300, with margin
    assert _charpoly_disc(ab - eps) > 0        # three distinct real eigenvalues below the bound
    assert _charpoly_disc(ab + eps) < 0        # a complex pair above it
    assert _charpoly_disc(ALPHA_PAPER) > 0


# ---------------------------------------------------------------------------
# Residual: exact-coefficient route vs brute-force quadrature.
# ---------------------------------------------------------------------------
def _chi_field(S, seed):
    """Per-site chi = -gamma_i (the appendix's m-site model), both signs."""
    return np.random.default_rng(seed).uniform(-2.0, 2.0, S)


@pytest.mark.parametrize("nx,ny,chi,eps0", [(4, 3, 1.3, 0.0), (5, 6, -0.7, 0.45), (5, 4, "field", 0.2)])
def test_residual_matches_brute_force_quadrature(nx, ny, chi, eps0):
    rng = np.random.default_rng(7)
    S = nx * ny
    if chi == "field":
        chi = _chi_field(S, 17)
    V = rng.uniform(-1, 1, S)
    tx, ty = 1.1, 0.8
    prob = orc.Problem(nx, ny, V, chi, tx=tx, ty=ty, eps0=eps0)
    u0 = _rand_state(rng, S)
    U = u0[None, :] + 0.1 * np.vstack([_rand_state(rng, S) for _ in range(3)])
    h = 0.03
    got = orc.residual(prob, u0, U, h)
    want = brute_phi(nx, ny, V, chi, tx, ty, eps0, u0, U, h)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(U))


def test_residual_matches_brute_force_quadrature_random_cases():
    """Property form of the pin above: random grid shapes (3..6 per side), hoppings of
    either sign, on-site shifts, chi (scalar or per site), step sizes and states; the
    oracle's exact-coefficient residual equals the 20-point brute-force quadrature of
    eq. (MB4_3) to rounding."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=25, deadline=None, derandomize=True)
    @hyp.given(nx=st.integers(3, 6), ny=st.integers(3, 6), tx=st.floats(-2, 2), ty=st.floats(-2, 2),
               eps0=st.floats(-1, 1), chi=st.floats(-3, 3), field=st.booleans(), h=st.floats(0.001, 0.1),
               seed=st.integers(0, 2 ** 31 - 1))
    def check(nx, ny, tx, ty, eps0, chi, field, h, seed):
        rng = np.random.default_rng(seed)
        S = nx * ny
        V = rng.uniform(-2, 2, S)
        c = rng.uniform(-3, 3, S) if field else chi
        prob = orc.Problem(nx, ny, V, c, tx=tx, ty=ty, eps0=eps0)
        u0 = _rand_state(rng, S)
        U = u0[None, :] + 0.2 * np.vstack([_rand_state(rng, S) for _ in range(3)])
        got = orc.residual(prob, u0, U, h)
        want = brute_phi(nx, ny, V, c, tx, ty, eps0, u0, U, h)
        assert np.max(np.abs(got - want)) <= 1e-13 * max(1.0, np.max(np.abs(U)) ** 3)

    check()


def test_residual_at_sites_matches_full_residual():
    rng = np.random.default_rng(3)
    nx, ny = 7, 5
    S = nx * ny
    V = rng.uniform(-1, 1, S)
    prob = orc.Problem(nx, ny, V, 0.9, tx=1.2, ty=0.6, eps0=0.3)
    u0 = _rand_state(rng, S)
    U = u0[None, :] + 0.1 * np.vstack([_rand_state(rng, S) for _ in range(3)])
    full = orc.residual(prob, u0, U, 0.02)
    sites = np.array([0, 6, 7, 17, 34, 28])
    part = orc.residual_at_sites(nx, ny, V, 0.9, 1.2, 0.6, 0.3, u0, U, 0.02, sites)
    assert np.max(np.abs(full[:, sites] - part)) <= 1e-15 * np.max(np.abs(U)) * 10


# ---------------------------------------------------------------------------
# Whole step.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("field", [False, True])
def test_step_matches_brute_force_root(field):
    """3x3 grid: the root of the brute-force Phi found by MINPACK (finite-difference
    Jacobian, no decoupling, no E) equals the oracle's Newton result; also with a
    per-site chi."""
    rng = np.random.default_rng(11)
    nx, ny = 3, 3
    S = nx * ny
    V = rng.uniform(-1, 1, S)
    V[4] += 5.0
    chi, tx, ty, eps0, h = 1.7, 1.0, 0.9, 0.2, 0.05
    if field:
        chi = _chi_field(S, 23)
    prob = orc.Problem(nx, ny, V, chi, tx=tx, ty=ty, eps0=eps0)
    u0 = _rand_state(rng, S, 0.5)
    u1_orc, U_orc, _ = orc.step(prob, u0, h, return_stages=True)

    def F(x):
        U = x[:3 * S] + 1j * x[3 * S:]
        Phi = brute_phi(nx, ny, V, chi, tx, ty, eps0, u0, U.reshape(3, S), h)
        return np.concatenate([Phi.real.ravel(), Phi.imag.ravel()])

    U0 = np.tile(u0, 3)
    sol = scipy.optimize.root(F, np.concatenate([U0.real, U0.imag]), method="hybr", tol=1e-15)
    Ub = (sol.x[:3 * S] + 1j * sol.x[3 * S:]).reshape(3, S)
    assert np.max(np.abs(F(sol.x))) < 1e-13
    assert np.max(np.abs(Ub - U_orc)) <= 1e-13 * np.max(np.abs(u0))


def test_quadrature_below_six_nodes_breaks_energy_preservation():
    """Negative control for the exact integration of the cubic term (Sec. 2.2): the stage
    integrand has degree 11 in zeta, so Gauss rules of 6 nodes integrate it exactly and of
    5 or 3 nodes (exact to degrees 9 and 5) do not.  Stages from the brute-force residual
    with each rule, solved by MINPACK on a 3x3 grid over 10 steps: 6 nodes keep H to the
    root finder's accuracy, 5 and 3 nodes lose it by orders of magnitude."""
    rng = np.random.default_rng(31)
    nx, ny = 3, 3
    S = nx * ny
    V = rng.uniform(-1, 1, S)
    chi, tx, ty, eps0, h = 2.0, 1.0, 0.9, 0.2, 0.1
    u0 = _rand_state(rng, S, 0.8)
    prob = orc.Problem(nx, ny, V, chi, tx=tx, ty=ty, eps0=eps0)
    drift = {}
    for nq in (6, 5, 3):
        u = u0.copy()
        H0 = orc.energy(prob, u)[0]
        d = 0.0
        for _ in range(10):
            def F(x, u=u):
                U = (x[:3 * S] + 1j * x[3 * S:]).reshape(3, S)
                P = brute_phi(nx, ny, V, chi, tx, ty, eps0, u, U, h, nq=nq)
                return np.concatenate([P.real.ravel(), P.imag.ravel()])
            U0 = np.tile(u, 3)
            sol = scipy.optimize.root(F, np.concatenate([U0.real, U0.imag]), method="hybr", tol=1e-15)
            assert np.max(np.abs(F(sol.x))) < 1e-12
            u = sol.x[2 * S:3 * S] + 1j * sol.x[5 * S:6 * S]
            d = max(d, abs(orc.energy(prob, u)[0] - H0) / abs(H0))
        drift[nq] = d
    assert drift[6] <= 1e-12, drift
    assert drift[5] >= 1e-6 and drift[3] >= 1e-6, drift


def _stability_function():
    """R(z) of MB4 from the continuous stage equation (eq. MB4_1) for u' = lambda u,
    u0 = 1: U_tau is a cubic in tau; equating coefficients gives R(z) = U_1
    (c3 = 1, B = A_1)."""
    sympy = pytest.importorskip("sympy")
    z, tau, zeta = sympy.symbols("z tau zeta")
    al = sympy.Rational(ALPHA_PAPER.numerator, ALPHA_PAPER.denominator)
    M = sympy.Matrix([[al + 4, -6 * al - 6, 6 * al],
                      [-6 * al - 6, 36 * al + 12, -36 * al],
                      [6 * al, -36 * al, 36 * al]])
    A = (sympy.Matrix([[tau, tau ** 2 / 2, tau ** 3 / 3]]) * M * sympy.Matrix([1, zeta, zeta ** 2]))[0]
    a = sympy.symbols("a1:4")
    Ut = lambda s: 1 + a[0] * s + a[1] * s ** 2 + a[2] * s ** 3
    rhs = 1 + z * sympy.integrate(A * Ut(zeta), (zeta, 0, 1))
    diff = sympy.Poly(sympy.expand(Ut(tau) - rhs), tau)
    sol = sympy.solve([diff.coeff_monomial(tau ** k) for k in (1, 2, 3)], a, dict=True)[0]
    R = sympy.simplify(Ut(1).subs(sol))
    return sympy, z, R


def test_stability_function_is_order4_and_unimodular():
    sympy, z, R = _stability_function()
    ser = sympy.series(R - sympy.exp(z), z, 0, 6).removeO()
    for k in range(5):
        assert sympy.simplify(ser.coeff(z, k)) == 0
    assert sympy.simplify(ser.coeff(z, 5)) != 0          # order exactly 4
    assert sympy.simplify(R * R.subs(z, -z) - 1) == 0     # |R(iy)| = 1: the norm is kept for chi = 0


def test_linear_step_equals_stability_function():
    """chi = 0: n oracle steps equal Q R(-i h Lambda)^n Q^H u0 with K+V = Q Lambda Q^H
    (dense eigendecomposition of a matrix built here by explicit loops)."""
    sympy, z, R = _stability_function()
    Rf = sympy.lambdify(z, R, "numpy")
    rng = np.random.default_rng(5)
    nx, ny, tx, ty, eps0 = 6, 5, 1.3, 0.7, 0.4
    S = nx * ny
    V = rng.uniform(-1, 1, S)
    V[7] = 20.0
    A = np.zeros((S, S))
    for y in range(ny):
        for x in range(nx):
            k = y * nx + x
            A[k, k] = eps0 + V[k]
            A[k, y * nx + (x + 1) % nx] -= tx
            A[k, y * nx + (x - 1) % nx] -= tx
            A[k, ((y + 1) % ny) * nx + x] -= ty
            A[k, ((y - 1) % ny) * nx + x] -= ty
    lam, Q = np.linalg.eigh(A)
    h, n = 0.01, 10
    u0 = _rand_state(rng, S)
    want = Q @ (Rf(-1j * h * lam) ** n * (Q.conj().T @ u0))
    prob = orc.Problem(nx, ny, V, 0.0, tx=tx, ty=ty, eps0=eps0)
    got, _ = orc.run(prob, u0, h, n)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(u0))
    assert abs(orc.norm2(got) - orc.norm2(u0)) <= 1e-13 * orc.norm2(u0)


def test_fourth_order_convergence_nonlinear():
    """chi != 0: error against a tight DOP853 reference falls by ~2^4 per halving of h."""
    rng = np.random.default_rng(9)
    nx, ny = 4, 3
    S = nx * ny
    V = rng.uniform(-1, 1, S)
    chi = 1.0
    prob = orc.Problem(nx, ny, V, chi, tx=1.0, ty=1.0, eps0=0.0)
    u0 = _rand_state(rng, S, 0.7)
    T = 0.4

    def rhs(t, y):
        u = y[:S] + 1j * y[S:]
        f = _f_roll(u, nx, ny, V, chi, 1.0, 1.0, 0.0)
        return np.concatenate([f.real, f.imag])

    ref = scipy.integrate.solve_ivp(rhs, (0, T), np.concatenate([u0.real, u0.imag]), method="DOP853",
                                    rtol=1e-13, atol=1e-14).y[:, -1]
    ref = ref[:S] + 1j * ref[S:]
    errs = []
    for n in (10, 20, 40):
        u, _ = orc.run(prob, u0, T / n, n)
        errs.append(np.max(np.abs(u - ref)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] > 3.8, (errs, rates)
    assert rates[0] > 3.5, (errs, rates)


def test_energy_preserved_grid16():
    """16x16 wavepacket workload, 100 steps: |dH/H| at the paper's 1e-14 level
    (we allow 1e-13), the norm to the paper's 1e-8."""
    w = inputs.grid16_fp64()
    prob = orc.Problem(w.nx, w.ny, w.potential(), w.chi, tx=w.tx, ty=w.ty, eps0=w.eps0)
    u = w.psi0()
    H0 = orc.energy(prob, u)[0]
    n0 = orc.norm2(u)
    drift = 0.0
    for _ in range(w.steps):
        u = orc.step(prob, u, w.h)
        drift = max(drift, abs(orc.energy(prob, u)[0] - H0) / abs(H0))
    assert drift <= 1e-13
    assert abs(orc.norm2(u) - n0) <= float(PAPER["norm_rel_drift_bound"][0])


def test_chi_field_energy_preserved_and_uniform_field_is_scalar():
    """The m-site model with site-dependent gamma_i is still of the form i u' =
    grad H, so MB4 keeps H = u^H (K+V) u + (1/2) sum chi_i |u_i|^4 to rounding; a
    uniform field gives the scalar-chi step bit for bit."""
    rng = np.random.default_rng(31)
    nx, ny = 8, 6
    S = nx * ny
    V = rng.uniform(-1, 1, S)
    chi = _chi_field(S, 37)
    prob = orc.Problem(nx, ny, V, chi, tx=1.1, ty=0.9, eps0=0.3)
    u = _rand_state(rng, S, 0.4)
    H0 = orc.energy(prob, u)[0]
    drift = 0.0
    for _ in range(30):
        u = orc.step(prob, u, 0.02)
        drift = max(drift, abs(orc.energy(prob, u)[0] - H0) / abs(H0))
    assert drift <= 1e-13, drift
    u0 = _rand_state(rng, S, 0.4)
    a = orc.step(orc.Problem(nx, ny, V, 1.3, tx=1.1, ty=0.9, eps0=0.3), u0, 0.02)
    b = orc.step(orc.Problem(nx, ny, V, np.full(S, 1.3), tx=1.1, ty=0.9, eps0=0.3), u0, 0.02)
    assert np.array_equal(a, b)


def _random_graph_K(S, deg, seed, onsite=0.3):
    """A random real symmetric site model: each site linked to up to deg others."""
    rng = np.random.default_rng(seed)
    K = np.zeros((S, S))
    for k in range(S):
        for j in rng.choice(S, size=deg // 2, replace=False):
            if j != k:
                w = rng.uniform(-1.5, 1.5)
                K[k, j] = K[j, k] = w
    return K + onsite * np.eye(S)


def _brute_phi_dense(K, V, chi, u0, U, h, nq=20):
    """Brute-force residual (20-point Gauss-Legendre of the stage integrals) for a dense K."""
    nodes = np.array([0.0] + [float(x) for x in C_PAPER])
    zq, wq = np.polynomial.legendre.leggauss(nq)
    zq, wq = 0.5 * (zq + 1.0), 0.5 * wq
    lag = scipy.interpolate.BarycentricInterpolator(nodes, np.eye(4))
    X = np.vstack([u0[None, :], U])
    acc = np.zeros_like(U)
    for z, w in zip(zq, wq):
        lz = lag(z)
        Uz = sum(lz[j] * X[j] for j in range(4))
        fz = -1j * (K @ Uz + V * Uz + chi * np.abs(Uz) ** 2 * Uz)
        for i in range(3):
            acc[i] += w * _A_float(ALPHA_PAPER, float(C_PAPER[i]), z) * fz
    return U - u0[None, :] - h * acc


def test_general_site_model():
    """A given kinetic matrix (the appendix's m-site model): the residual equals the
    brute-force quadrature with a dense K, energy is conserved, and the 5-point
    stencil handed over as a matrix reproduces the grid problem bit for bit."""
    rng = np.random.default_rng(43)
    S = 30
    K = _random_graph_K(S, 6, 44)
    V = rng.uniform(-1, 1, S)
    chi = _chi_field(S, 45)
    prob = orc.Problem.general(K, V, chi)
    u0 = _rand_state(rng, S, 0.5)
    U = u0[None, :] + 0.1 * np.vstack([_rand_state(rng, S) for _ in range(3)])
    got = orc.residual(prob, u0, U, 0.03)
    want = _brute_phi_dense(K, V, chi, u0, U, 0.03)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(U))
    u, H0, drift = u0, orc.energy(prob, u0)[0], 0.0
    for _ in range(30):
        u = orc.step(prob, u, 0.02)
        drift = max(drift, abs(orc.energy(prob, u)[0] - H0) / abs(H0))
    assert drift <= 1e-13, drift
    nx, ny = 5, 4
    grid = orc.Problem(nx, ny, V[:20], 1.1, tx=1.2, ty=0.8, eps0=0.3)
    gen = orc.Problem.general(grid.K, V[:20], 1.1)
    w0 = _rand_state(rng, nx * ny, 0.5)
    assert np.array_equal(orc.step(grid, w0, 0.02), orc.step(gen, w0, 0.02))


def test_time_reversal():
    """MB4 is symmetric: a step of -h undoes a step of h."""
    rng = np.random.default_rng(1)
    nx, ny = 6, 5
    S = nx * ny
    V = rng.uniform(-1, 1, S)
    prob = orc.Problem(nx, ny, V, 1.0, tx=1.3, ty=0.7, eps0=0.4)
    u0 = _rand_state(rng, S)
    back = orc.step(prob, orc.step(prob, u0, 0.02), -0.02)
    assert np.max(np.abs(back - u0)) <= 1e-14 * np.max(np.abs(u0))


def test_translation_and_transpose_equivariance():
    rng = np.random.default_rng(2)
    nx = ny = 6
    S = nx * ny
    V = rng.uniform(-1, 1, S)
    u0 = _rand_state(rng, S)
    prob = orc.Problem(nx, ny, V, 1.1, tx=1.0, ty=1.0, eps0=0.2)
    u1 = orc.step(prob, u0, 0.03).reshape(ny, nx)
    roll = lambda a: np.roll(np.roll(a.reshape(ny, nx), 2, axis=1), -1, axis=0)
    prob_r = orc.Problem(nx, ny, roll(V).ravel(), 1.1, tx=1.0, ty=1.0, eps0=0.2)
    u1r = orc.step(prob_r, roll(u0).ravel(), 0.03)
    assert np.max(np.abs(u1r - roll(u1).ravel())) <= 1e-14 * np.max(np.abs(u0))
    tr = lambda a: a.reshape(ny, nx).T.copy()
    prob_t = orc.Problem(nx, ny, tr(V).ravel(), 1.1, tx=1.0, ty=1.0, eps0=0.2)
    u1t = orc.step(prob_t, tr(u0).ravel(), 0.03)
    assert np.max(np.abs(u1t - u1.T.ravel())) <= 1e-14 * np.max(np.abs(u0))


def test_plane_wave_keeps_modulus():
    """psi = a exp(i k.x) with constant V stays a plane wave with |a| kept: the
    flow is a' = -i(e_k + V + chi |a|^2) a and MB4 preserves the per-site
    energy, which fixes |a|."""
    nx, ny = 8, 6
    S = nx * ny
    kx, ky = 2 * math.pi * 3 / nx, 2 * math.pi * 1 / ny
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    a = 0.8 * np.exp(0.3j)
    u0 = (a * np.exp(1j * (kx * x + ky * y))).ravel()
    prob = orc.Problem(nx, ny, np.full(S, 0.7), 1.5, tx=1.0, ty=0.5, eps0=0.1)
    u = u0
    for _ in range(5):
        u = orc.step(prob, u, 0.05)
    ratio = u / u0
    assert np.max(np.abs(ratio - ratio[0])) < 1e-14
    assert abs(abs(ratio[0]) - 1.0) < 1e-14


def test_splitmix64_reference_outputs():
    want = [int(x, 16) for x in TEXTBOOK["splitmix64_seed0"]]
    got = [int(v) for v in inputs.splitmix64(0, 3)]
    assert got == want


def test_inputs_shapes_and_normalisation():
    w = inputs.grid16_fp64()
    V = w.potential()
    assert V.shape == (256,)
    assert np.sum(V > 10) == 3
    psi = w.psi0()
    assert abs(orc.norm2(psi) - 1.0) < 1e-15
    w2 = inputs.grid512_fp64()
    assert w2.defects() == round(0.01 * 512 * 512)


@pytest.mark.parametrize("field", [False, True])
def test_jacobian_matches_finite_difference(field):
    """J of eq. (JL) + eq. (JR) (real form, gamma = -chi) against central differences
    of the brute-force f.  J only steers the simplified Newton iteration, so a
    wrong J would not move the root; this pins it directly (also per-site chi)."""
    rng = np.random.default_rng(4)
    nx, ny = 4, 3
    S = nx * ny
    V = rng.uniform(-1, 1, S)
    chi, tx, ty, eps0 = 1.4, 1.2, 0.7, 0.3
    if field:
        chi = _chi_field(S, 29)
    prob = orc.Problem(nx, ny, V, chi, tx=tx, ty=ty, eps0=eps0)
    u0 = _rand_state(rng, S)
    J = orc.jacobian_real(prob, u0).toarray()

    def freal(x):
        f = _f_roll(x[:S] + 1j * x[S:], nx, ny, V, chi, tx, ty, eps0)
        return np.concatenate([f.real, f.imag])

    x0 = np.concatenate([u0.real, u0.imag])
    d = 1e-6
    Jfd = np.zeros((2 * S, 2 * S))
    for k in range(2 * S):
        e = np.zeros(2 * S)
        e[k] = d
        Jfd[:, k] = (freal(x0 + e) - freal(x0 - e)) / (2 * d)
    assert np.max(np.abs(J - Jfd)) < 1e-7 * max(1.0, np.max(np.abs(J)))


def test_oracle_linear_solvers_agree():
    """The oracle's two Newton linear solvers (sparse LU, GMRES on the coupled
    matrix) reach the same root of Phi(U) = 0."""
    w = inputs.grid512_fp64()
    n = 24
    V = inputs.potential(n, n, 1.0, 6, 20.0, 3)
    prob = orc.Problem(n, n, V, 1.0)
    u0 = inputs.wavepacket(n, n, 3.0, math.pi / 4, 0.0)
    ul, _ = orc.run(prob, u0, w.h, 3, solver="lu")
    ug, _ = orc.run(prob, u0, w.h, 3, solver="gmres")
    assert np.max(np.abs(ul - ug)) <= 1e-15 * np.max(np.abs(ul))


# ---------------------------------------------------------------------------
# Observables: the split of H into U_K, U_E, U_I (Sec. 2.1, eq. U_K .. U_E) and the
# participation ratio p = sum |u|^4 (Sec. 3.2), pinned by closed forms, by special
# states and by an independent Fourier route -- not by the oracle's own formulas.
# ---------------------------------------------------------------------------
def _plane_wave(nx, ny, mx, my, a):
    kx, ky = 2 * math.pi * mx / nx, 2 * math.pi * my / ny
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    return (a * np.exp(1j * (kx * x + ky * y))).ravel(), kx, ky


@pytest.mark.parametrize("field", [False, True])
def test_observables_of_a_plane_wave(field):
    """psi = a exp(i k.x) is an eigenvector of the 5-point K with eigenvalue
    eps0 - 2 tx cos kx - 2 ty cos ky, and |psi|^2 = |a|^2 at every site, so
    U_K = S |a|^2 (eps0 - 2 tx cos kx - 2 ty cos ky), U_E = |a|^2 sum_k V_k (for any V),
    U_I = (|a|^4 / 2) sum_k chi_k, sum |u|^2 = S |a|^2 and p = S |a|^4."""
    rng = np.random.default_rng(71)
    nx, ny = 7, 5
    S = nx * ny
    tx, ty, eps0 = 1.3, -0.6, 0.45
    V = rng.uniform(-2, 3, S)
    chi = _chi_field(S, 72) if field else 1.7
    chis = np.broadcast_to(chi, (S,))
    a = 0.37 * np.exp(0.8j)
    u, kx, ky = _plane_wave(nx, ny, 2, 3, a)
    prob = orc.Problem(nx, ny, V, chi, tx=tx, ty=ty, eps0=eps0)
    H, UK, UE, UI = orc.energy(prob, u)
    A2 = abs(a) ** 2
    want_K = S * A2 * (eps0 - 2 * tx * math.cos(kx) - 2 * ty * math.cos(ky))
    want_E = A2 * math.fsum(V.tolist())
    want_I = 0.5 * A2 * A2 * math.fsum(chis.tolist())
    for got, want in ((UK, want_K), (UE, want_E), (UI, want_I), (H, want_K + want_E + want_I)):
        assert abs(got - want) <= 1e-14 * (abs(want_K) + abs(want_E) + abs(want_I)), (got, want)
    assert abs(orc.norm2(u) - S * A2) <= 1e-15 * S * A2
    assert abs(orc.participation(u) - S * A2 * A2) <= 1e-15 * S * A2 * A2


def test_kinetic_energy_by_parseval():
    """The 5-point K is diagonal in Fourier space, so for ANY state
    U_K = (1/S) sum_m eps_m |uhat_m|^2 with uhat the 2D DFT of u and
    eps_m = eps0 - 2 tx cos(2 pi mx / nx) - 2 ty cos(2 pi my / ny); likewise
    sum |u|^2 = (1/S) sum |uhat|^2 (Parseval).  A route through numpy's FFT that
    shares nothing with the oracle's sparse K."""
    rng = np.random.default_rng(73)
    nx, ny = 9, 6
    S = nx * ny
    tx, ty, eps0 = 0.8, 1.9, -0.3
    V = rng.uniform(-1, 1, S)
    u = _rand_state(rng, S, 0.3)
    prob = orc.Problem(nx, ny, V, 1.1, tx=tx, ty=ty, eps0=eps0)
    uh = np.fft.fft2(u.reshape(ny, nx))
    mx = np.arange(nx)[None, :]
    my = np.arange(ny)[:, None]
    eps = eps0 - 2 * tx * np.cos(2 * math.pi * mx / nx) - 2 * ty * np.cos(2 * math.pi * my / ny)
    want_K = float(np.sum(eps * np.abs(uh) ** 2)) / S
    _, UK, _, _ = orc.energy(prob, u)
    assert abs(UK - want_K) <= 1e-13 * float(np.sum(np.abs(eps) * np.abs(uh) ** 2)) / S
    assert abs(orc.norm2(u) - float(np.sum(np.abs(uh) ** 2)) / S) <= 1e-13 * orc.norm2(u)


def test_observables_of_a_site_state():
    """u = c e_j (all weight on site j): U_K = eps0 |c|^2 (K's diagonal), U_E = V_j |c|^2,
    U_I = (chi_j / 2) |c|^4, p = |c|^4 -- each term picks out its own coefficient, so a
    term assigned to the wrong part, or a wrong power of |u|, changes the numbers."""
    rng = np.random.default_rng(74)
    nx, ny = 5, 4
    S = nx * ny
    V = rng.uniform(-3, 3, S)
    chi = _chi_field(S, 75)
    prob = orc.Problem(nx, ny, V, chi, tx=0.9, ty=1.4, eps0=0.65)
    c = 0.6 - 0.5j
    n = abs(c) ** 2
    for j in (0, 7, S - 1):
        u = np.zeros(S, dtype=np.complex128)
        u[j] = c
        H, UK, UE, UI = orc.energy(prob, u)
        assert abs(UK - 0.65 * n) <= 1e-15
        assert abs(UE - V[j] * n) <= 1e-15 * max(1.0, abs(V[j]))
        assert abs(UI - 0.5 * chi[j] * n * n) <= 1e-15
        assert abs(H - (0.65 + V[j]) * n - 0.5 * chi[j] * n * n) <= 1e-14
        assert abs(orc.participation(u) - n * n) <= 1e-16
        assert abs(orc.norm2(u) - n) <= 1e-16


def test_participation_ratio_of_spread_states():
    """Sec. 3.2: p = sum |u|^4 equals 1/(Nx Ny) for a normalised state of uniform
    density (the paper's own value, 1e-4 on its 100 x 100 grid) and grows as the
    state localises: 1/M for a normalised state spread evenly over M sites, 1 on one
    site.  sum |u|^2 is 1 in every case, so p is not the norm."""
    rng = np.random.default_rng(76)
    nx = ny = 100
    S = nx * ny
    phase = np.exp(2j * math.pi * rng.uniform(size=S))
    uniform = phase / math.sqrt(S)
    assert abs(orc.participation(uniform) - 1e-4) <= 1e-17
    for M in (1, 3, 250):
        u = np.zeros(S, dtype=np.complex128)
        sites = rng.choice(S, size=M, replace=False)
        u[sites] = phase[sites] / math.sqrt(M)
        assert abs(orc.norm2(u) - 1.0) <= 1e-15
        assert abs(orc.participation(u) - 1.0 / M) <= 1e-15 / M


# ---------------------------------------------------------------------------
# Complex Hermitian K (the appendix's m-site model with complex transfer integrals;
# Sec. 2.1 asks only that K be Hermitian).
# ---------------------------------------------------------------------------
def _random_hermitian_K(S, deg, seed, onsite=0.3):
    """A random sparse Hermitian site model: links t e^{i phi} (Peierls-like phases)."""
    rng = np.random.default_rng(seed)
    K = np.zeros((S, S), dtype=np.complex128)
    for k in range(S):
        for j in rng.choice(S, size=deg // 2, replace=False):
            if j != k:
                w = rng.uniform(-1.5, 1.5) * np.exp(1j * rng.uniform(-math.pi, math.pi))
                K[k, j] = w
                K[j, k] = np.conj(w)
    return K + onsite * np.eye(S)


def _f_dense(K, V, chi, u):
    return -1j * (K @ u + V * u + chi * np.abs(u) ** 2 * u)


def test_complex_hermitian_site_model_residual_and_energy():
    """With a complex Hermitian K the oracle's residual equals the brute-force
    quadrature of eq. (MB4_3), and MB4 keeps H = u^H (K+V) u + (1/2) sum chi |u|^4 (real
    for Hermitian K) to rounding over 30 steps."""
    rng = np.random.default_rng(81)
    S = 28
    K = _random_hermitian_K(S, 6, 82)
    V = rng.uniform(-1, 1, S)
    chi = _chi_field(S, 83)
    prob = orc.Problem.general(K, V, chi)
    assert np.iscomplexobj(prob.A.data)
    u0 = _rand_state(rng, S, 0.5)
    U = u0[None, :] + 0.1 * np.vstack([_rand_state(rng, S) for _ in range(3)])
    got = orc.residual(prob, u0, U, 0.03)
    want = _brute_phi_dense(K, V, chi, u0, U, 0.03)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(U))
    u, H0, drift = u0, orc.energy(prob, u0)[0], 0.0
    want_H = float(np.real(np.vdot(u0, (K + np.diag(V)) @ u0))) + 0.5 * float(np.sum(chi * np.abs(u0) ** 4))
    assert abs(H0 - want_H) <= 1e-13 * abs(H0)
    for _ in range(30):
        u = orc.step(prob, u, 0.02)
        drift = max(drift, abs(orc.energy(prob, u)[0] - H0) / abs(H0))
    assert drift <= 1e-13, drift


def test_complex_hermitian_jacobian_matches_finite_difference():
    """The real form of J with a complex A = K + V ([[Im A, Re A], [-Re A, Im A]] plus
    eq. (JR)) against central differences of f(u) = -i[(K+V)u + chi|u|^2 u]."""
    rng = np.random.default_rng(84)
    S = 10
    K = _random_hermitian_K(S, 4, 85)
    V = rng.uniform(-1, 1, S)
    chi = 1.3
    prob = orc.Problem.general(K, V, chi)
    u0 = _rand_state(rng, S)
    J = orc.jacobian_real(prob, u0).toarray()

    def freal(x):
        f = _f_dense(K, V, chi, x[:S] + 1j * x[S:])
        return np.concatenate([f.real, f.imag])

    x0 = np.concatenate([u0.real, u0.imag])
    d = 1e-6
    Jfd = np.zeros((2 * S, 2 * S))
    for k in range(2 * S):
        e = np.zeros(2 * S)
        e[k] = d
        Jfd[:, k] = (freal(x0 + e) - freal(x0 - e)) / (2 * d)
    assert np.max(np.abs(J - Jfd)) < 1e-7 * max(1.0, np.max(np.abs(J)))


def test_gauge_transformed_kinetic_matrix_gives_the_gauge_transformed_step():
    """A site-dependent phase G = diag(e^{i theta_k}) is a symmetry of the equation:
    |G u|^2 = |u|^2 and V is diagonal, so with K' = G K G^H the flow maps G u0 to
    G u(t), and MB4 (affine-covariant, like every Runge-Kutta method) maps G u0 to
    G u1.  K' is complex although K -- here the grid stencil -- is real, so this ties
    the complex-K route to the real one."""
    rng = np.random.default_rng(86)
    nx, ny = 5, 4
    S = nx * ny
    V = rng.uniform(-1, 1, S)
    grid = orc.Problem(nx, ny, V, 1.2, tx=1.1, ty=0.7, eps0=0.3)
    theta = rng.uniform(-math.pi, math.pi, S)
    G = np.exp(1j * theta)
    Kc = (G[:, None] * grid.K.toarray()) * np.conj(G)[None, :]
    Kc = 0.5 * (Kc + Kc.conj().T)          # Hermitian to the last bit (the products round)
    gauge = orc.Problem.general(Kc, V, 1.2)
    u0 = _rand_state(rng, S, 0.5)
    u1 = orc.step(grid, u0, 0.02)
    u1g = orc.step(gauge, G * u0, 0.02)
    assert np.max(np.abs(u1g - G * u1)) <= 1e-14 * np.max(np.abs(u0))


def test_linear_complex_K_step_equals_stability_function():
    """chi = 0 with a complex Hermitian K: n steps equal Q R(-i h Lambda)^n Q^H u0 with
    K + V = Q Lambda Q^H, and the norm is kept (|R(iy)| = 1)."""
    sympy, z, R = _stability_function()
    Rf = sympy.lambdify(z, R, "numpy")
    rng = np.random.default_rng(87)
    S = 24
    K = _random_hermitian_K(S, 6, 88)
    V = rng.uniform(-1, 1, S)
    lam, Q = np.linalg.eigh(K + np.diag(V))
    h, n = 0.02, 8
    u0 = _rand_state(rng, S)
    want = Q @ (Rf(-1j * h * lam) ** n * (Q.conj().T @ u0))
    got, _ = orc.run(orc.Problem.general(K, V, 0.0), u0, h, n)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(u0))
    assert abs(orc.norm2(got) - orc.norm2(u0)) <= 1e-13 * orc.norm2(u0)


def test_general_rejects_a_non_hermitian_K():
    K = _random_hermitian_K(8, 4, 89)
    K[0, 1] += 0.1j
    with pytest.raises(ValueError):
        orc.Problem.general(K, np.zeros(8), 1.0)
