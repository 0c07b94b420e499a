"""Planted mistakes in the oracle, each caught by a pin.

Every test here swaps one function of the oracle for a copy with one plausible
mistake (a flipped sign, a dropped term, a missing conjugate, swapped hoppings, the
wrong stage, a loose stopping rule) and runs the pin of test_oracle_pins.py that
should catch it: the pin must fail.  This shows the pins constrain the oracle from
outside its own arithmetic.  CPU only; the oracle is restored after each test.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import mb4_oracle as orc

import test_oracle_pins as pins


@pytest.fixture(autouse=True)
def _fresh_constants():
    orc.mb4_constants.cache_clear()
    yield
    orc.mb4_constants.cache_clear()


def _fails(pin, *args):
    """True if the pin raises (an assertion, or an error of the mutated oracle)."""
    try:
        pin(*args)
    except Exception:
        return True
    return False


# ---------------------------------------------------------------------------
# Constants.
# ---------------------------------------------------------------------------
def test_sign_in_the_mb4_matrix(monkeypatch):
    """eq. (Adefinition) with the (1, 2) entry's sign flipped."""
    good = orc.mb4_matrix

    def bad(alpha1):
        M = good(alpha1)
        M[0][1] = -M[0][1]
        return M
    monkeypatch.setattr(orc, "mb4_matrix", bad)
    assert _fails(pins.test_E_row_sums_are_the_nodes) or _fails(pins.test_last_row_of_E_is_simpson_three_eighths)


def test_lagrange_nodes_in_the_wrong_order(monkeypatch):
    """eq. (Lagrange) built on (c1, c2, c3, 0) instead of (0, c1, c2, c3)."""
    good = orc.lagrange_basis
    monkeypatch.setattr(orc, "lagrange_basis", lambda nodes: good(tuple(nodes[1:]) + (nodes[0],)))
    assert _fails(pins.test_last_row_of_E_is_simpson_three_eighths)


# ---------------------------------------------------------------------------
# Residual.
# ---------------------------------------------------------------------------
def _residual_variant(drop_cubic=False, no_conj=False, drop_e0=False):
    def residual(prob, u0, U, h, alpha1=orc.ALPHA1_PAPER, c=orc.C_PAPER):
        E, C3 = orc.constants_f64(alpha1, c)
        u0 = np.asarray(u0, dtype=np.complex128)
        U = np.asarray(U, dtype=np.complex128)
        X = np.vstack([u0[None, :], U])
        Y = (E[:, 1:] @ U) if drop_e0 else (E @ X)
        lin = -1j * np.vstack([prob.A @ Y[i] for i in range(3)])
        if drop_cubic:
            cub = 0.0
        elif no_conj:                                    # u^3 instead of |u|^2 u
            cub = -1j * prob.chi * np.einsum("iabd,ak,bk,dk->ik", C3, X, X, X)
        else:
            cub = -1j * prob.chi * np.einsum("iabd,ak,bk,dk->ik", C3, np.conj(X), X, X)
        return U - u0[None, :] - h * (lin + cub)
    return residual


@pytest.mark.parametrize("mistake", ["drop_cubic", "no_conj", "drop_e0"])
def test_residual_mistakes(monkeypatch, mistake):
    """eq. (fIu2) dropped or without its conjugate (u^3 for |u|^2 u), or eq. (fKu2)
    without the E_i0 u0 term: the brute-force quadrature of eq. (MB4_3) disagrees.  (The
    conjugate on another factor would be no mistake: the cubic coefficients are symmetric
    in their three indices.)"""
    monkeypatch.setattr(orc, "residual", _residual_variant(**{mistake: True}))
    assert _fails(pins.test_residual_matches_brute_force_quadrature, 4, 3, 1.3, 0.0)


def test_hoppings_swapped_in_the_kinetic_matrix(monkeypatch):
    """eq. (Kdefinition) with the x and y Kronecker factors exchanged (tx != ty)."""
    def bad(nx, ny, tx, ty, eps0):
        Ix = sp.identity(nx, format="csr")
        Iy = sp.identity(ny, format="csr")
        K = (-ty * sp.kron(Iy, orc._circulant_adjacency(nx))
             - tx * sp.kron(orc._circulant_adjacency(ny), Ix)
             + eps0 * sp.identity(nx * ny))
        return sp.csr_matrix(K)
    monkeypatch.setattr(orc, "kinetic_matrix", bad)
    assert _fails(pins.test_residual_matches_brute_force_quadrature, 5, 6, -0.7, 0.45)


# ---------------------------------------------------------------------------
# Jacobian, step, energy.
# ---------------------------------------------------------------------------
def test_sign_in_the_cubic_jacobian(monkeypatch):
    """eq. (JR) with the sign of its (2, 1) block flipped."""
    def bad(prob, u0):
        p0, q0 = np.real(u0), np.imag(u0)
        g = -prob.chi * np.ones_like(p0)
        JL = sp.bmat([[None, prob.A], [-prob.A, None]])
        JI = sp.bmat([[sp.diags(-2 * g * p0 * q0), sp.diags(-g * (p0 ** 2 + 3 * q0 ** 2))],
                      [sp.diags(-g * (3 * p0 ** 2 + q0 ** 2)), sp.diags(2 * g * p0 * q0)]])
        return sp.csr_matrix(JL + JI)
    monkeypatch.setattr(orc, "jacobian_real", bad)
    assert _fails(pins.test_jacobian_matches_finite_difference, False)


def test_step_returns_the_first_stage(monkeypatch):
    """u1 taken as U_c1 instead of U_c3 (Sec. 2.2, c3 = 1)."""
    good = orc.step

    def bad(prob, u0, h, **kw):
        want_stages = kw.pop("return_stages", False)
        u1, U, it = good(prob, u0, h, return_stages=True, **kw)
        return (U[0].copy(), U, it) if want_stages else U[0].copy()
    monkeypatch.setattr(orc, "step", bad)
    assert _fails(pins.test_linear_step_equals_stability_function)


def test_loose_newton_stopping_rule(monkeypatch):
    """Algorithm 1's test with a tolerance 1e6 times too loose."""
    good = orc.step
    monkeypatch.setattr(orc, "step", lambda prob, u0, h, **kw: good(prob, u0, h, **{**kw, "tol": 1e-8}))
    assert _fails(pins.test_step_matches_brute_force_root, False)


def test_energy_without_the_half(monkeypatch):
    """U_I with chi sum |u|^4 instead of (chi/2) sum |u|^4 (Sec. 2.1): not the
    conserved quantity, so the energy pin fails."""
    def bad(prob, u):
        u = np.asarray(u, dtype=np.complex128)
        tK = np.real(np.conj(u) * (prob.K @ u))
        n = np.abs(u) ** 2
        tE = prob.V * n
        tI = prob.chi * n * n
        H = float(np.sum(tK) + np.sum(tE) + np.sum(tI))
        return H, float(np.sum(tK)), float(np.sum(tE)), float(np.sum(tI))
    monkeypatch.setattr(orc, "energy", bad)
    assert _fails(pins.test_energy_preserved_grid16)


def test_kinetic_and_potential_energy_swapped(monkeypatch):
    """energy() returning U_E in the place of U_K and U_K in the place of U_E (their
    sum, H, unchanged -- so energy conservation alone cannot see it)."""
    good = orc.energy

    def bad(prob, u):
        H, UK, UE, UI = good(prob, u)
        return H, UE, UK, UI
    monkeypatch.setattr(orc, "energy", bad)
    assert _fails(pins.test_energy_preserved_grid16) is False      # H is still conserved
    assert _fails(pins.test_observables_of_a_plane_wave, False)
    assert _fails(pins.test_observables_of_a_site_state)


def test_participation_with_the_wrong_power(monkeypatch):
    """p = sum |u|^2 (the norm) instead of sum |u|^4 (Sec. 3.2)."""
    monkeypatch.setattr(orc, "participation", lambda u: orc.norm2(u))
    assert _fails(pins.test_participation_ratio_of_spread_states)
    assert _fails(pins.test_observables_of_a_plane_wave, True)


def test_factor_moved_between_energy_parts(monkeypatch):
    """A factor moved from U_I to U_E (chi/2 |u|^4 counted with the potential term),
    again with H unchanged."""
    good = orc.energy

    def bad(prob, u):
        H, UK, UE, UI = good(prob, u)
        return H, UK, UE + UI, 0.0
    monkeypatch.setattr(orc, "energy", bad)
    assert _fails(pins.test_observables_of_a_site_state)


def test_complex_jacobian_with_the_imaginary_blocks_flipped(monkeypatch):
    """The real form of J for a complex A = K + V with the sign of its Im A blocks flipped
    ([[-Im A, Re A], [-Re A, -Im A]]): the finite-difference pin with a complex K fails."""
    good = orc.jacobian_real

    def bad(prob, u0):
        J = good(prob, u0)
        if not np.iscomplexobj(prob.A.data):
            return J
        Ai = sp.csr_matrix(prob.A.imag)
        return sp.csr_matrix(J - 2 * sp.bmat([[Ai, None], [None, Ai]]))
    monkeypatch.setattr(orc, "jacobian_real", bad)
    assert _fails(pins.test_complex_hermitian_jacobian_matches_finite_difference)


def test_kinetic_matrix_taken_transposed(monkeypatch):
    """Problem.general storing K^T (= conj K for a Hermitian K) instead of K: the phases
    act backwards, the gauge pin and the brute-force residual with a complex K fail."""
    good = orc.Problem.general.__func__

    def bad(cls, K, V, chi):
        return good(cls, sp.csr_matrix(K).T, V, chi)
    monkeypatch.setattr(orc.Problem, "general", classmethod(bad))
    assert _fails(pins.test_gauge_transformed_kinetic_matrix_gives_the_gauge_transformed_step)
    assert _fails(pins.test_complex_hermitian_site_model_residual_and_energy)


def test_unmutated_oracle_passes_the_same_pins():
    """The control: with the oracle as it stands, every pin used above passes."""
    pins.test_E_row_sums_are_the_nodes()
    pins.test_last_row_of_E_is_simpson_three_eighths()
    pins.test_residual_matches_brute_force_quadrature(4, 3, 1.3, 0.0)
    pins.test_residual_matches_brute_force_quadrature(5, 6, -0.7, 0.45)
    pins.test_jacobian_matches_finite_difference(False)
    pins.test_step_matches_brute_force_root(False)
    pins.test_energy_preserved_grid16()
    pins.test_linear_step_equals_stability_function()
    pins.test_observables_of_a_plane_wave(False)
    pins.test_observables_of_a_plane_wave(True)
    pins.test_observables_of_a_site_state()
    pins.test_participation_ratio_of_spread_states()
    pins.test_complex_hermitian_jacobian_matches_finite_difference()
    pins.test_gauge_transformed_kinetic_matrix_gives_the_gauge_transformed_step()
    pins.test_complex_hermitian_site_model_residual_and_energy()
    assert Fraction(orc.C_PAPER[2]) == 1
