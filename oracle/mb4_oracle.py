"""Plain FP64 CPU oracle for one MB4 time step of the discrete NLS-type system.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only the tests, the smoke check and the benchmark's CPU
baseline leg use it.  It shares no code with the CUDA path and imports nothing
from the package.

What it computes (Sakai, Kudo, Imachi, Miyatake, Hoshi, Yamamoto,
"A parallelizable energy-preserving integrator MB4 and its application to
quantum-mechanical wavepacket dynamics", arXiv:2003.04345):

* The system is eq. (dNLS): i du/dt = K u - gamma (conj(u) o u) o u + V u on an
  Nx x Ny periodic grid, site index k = y*Nx + x (x fastest, Sec. 2.1).  We
  write chi = -gamma (Table 2 calls it ``eps``), so
      f(u) = -i [ (K + V) u + chi |u|^2 u ].
  K is eq. (Kdefinition), generalised to a hopping tx, ty and an on-site shift
  eps0:  K = -tx (I_Ny (x) C_Nx) - ty (C_Ny (x) I_Nx) + eps0 I,  with C_N the
  periodic adjacency (zero diagonal, ones at +-1).  The paper's Laplacian is
  tx = 1/hx^2, ty = 1/hy^2, eps0 = 2 tx + 2 ty.  Problem.general takes any Hermitian
  K instead (the appendix's m-site model; complex transfer integrals such as Peierls
  phases included): the paper needs only that K be Hermitian (Sec. 2.1).
* The MB4 coefficients are eq. (Adefinition); the stage polynomial is written
  in Lagrange form on c0 = 0, c1, c2, c3 (eq. Lagrange), and the stage
  equations are Phi(U) = 0 (eq. MB4_3, eq. Phidefinition).  With c3 = 1 the
  step result is u1 = U_c3 (Sec. 2.2, last paragraph).
* The linear part of the stage integrals is eq. (fKu2) with the constants
  E_ij, E_i0 of eq. (defE), eq. (Ei0).  The cubic part is eq. (fIu2): a
  homogeneous cubic in u0, U_c1..U_c3 and their conjugates whose coefficients
  are definite integrals of degree-11 polynomials.  Here those coefficients are
  computed exactly in rational arithmetic (the paper used Maxima, Sec. 3).
* The nonlinear system is solved by the simplified Newton iteration of
  eq. (Newton1) on the COUPLED 3N system (I - h E (x) J) r = -Phi, with J the
  real-form Jacobian of eq. (JL) + eq. (JR) frozen at u0 (eq. Jacobian2).  The
  eigen-decoupling of eq. (Newton3) is deliberately not used, so that the GPU
  path's decoupled solves are checked against an independent route.  Each
  linear solve is a sparse direct LU (SuperLU via scipy), like the paper's use
  of a sparse direct solver (Sec. 3.2), for grids of up to 1024 sites; above
  that, where the LU fill-in makes it slow, scipy's restarted GMRES on the same
  coupled matrix to a relative residual of 1e-13.  The solver changes only how
  fast the Newton iteration reaches the root of Phi(U) = 0, not the root.
* Energy H = u^H K u + u^H V u + (chi/2) sum |u|^4 (Sec. 2.1, U_K + U_E + U_I)
  and the norm sum |u|^2 are summed with math.fsum (correctly rounded).
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# Paper defaults (Sec. 3, parameter list): alpha1 = -300*19/8, c = (1/3, 2/3, 1).
ALPHA1_PAPER = Fraction(-300 * 19, 8)
C_PAPER = (Fraction(1, 3), Fraction(2, 3), Fraction(1))


# ---------------------------------------------------------------------------
# Exact polynomial algebra (coefficient lists, lowest degree first).
# ---------------------------------------------------------------------------
def _pmul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x == 0:
            continue
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _pint01(a):
    """Exact integral over [0, 1] of the polynomial a."""
    return sum((x / (k + 1) for k, x in enumerate(a)), Fraction(0))


def _peval(a, z):
    acc = Fraction(0)
    for x in reversed(a):
        acc = acc * z + x
    return acc


def mb4_matrix(alpha1):
    """The 3x3 matrix in the middle of eq. (Adefinition)."""
    a = Fraction(alpha1)
    return [[a + 4, -6 * a - 6, 6 * a],
            [-6 * a - 6, 36 * a + 12, -36 * a],
            [6 * a, -36 * a, 36 * a]]


def A_poly_in_zeta(alpha1, tau):
    """A_{tau, zeta} as a polynomial in zeta (degree 2), eq. (Adefinition):
    A = [tau, tau^2/2, tau^3/3] M [1, zeta, zeta^2]^T."""
    M = mb4_matrix(alpha1)
    tau = Fraction(tau)
    row = [tau, tau ** 2 / 2, tau ** 3 / 3]
    return [sum((row[a] * M[a][b] for a in range(3)), Fraction(0)) for b in range(3)]


def lagrange_basis(nodes):
    """l_j(zeta) with l_j(c_m) = delta_jm on the nodes (c0=0, c1, c2, c3), eq. (Lagrange)."""
    nodes = [Fraction(x) for x in nodes]
    basis = []
    for j, cj in enumerate(nodes):
        p = [Fraction(1)]
        for m, cm in enumerate(nodes):
            if m == j:
                continue
            p = _pmul(p, [-cm / (cj - cm), Fraction(1) / (cj - cm)])
        basis.append(p)
    return basis


@lru_cache(maxsize=16)
def mb4_constants(alpha1=ALPHA1_PAPER, c=C_PAPER):
    """Exact MB4 constants for the given alpha1 and (c1, c2, c3).

    Returns a dict with
      E   : 3x4 list of Fractions, E[i-1][j] = int_0^1 A_{c_i,zeta} l_j(zeta) dzeta
            for i = 1..3, j = 0..3 (j = 0 is E_i0 of eq. (Ei0), j >= 1 is eq. (defE));
      C3  : 3x4x4x4 nested list, C3[i-1][a][b][d] = int_0^1 A_{c_i,zeta} l_a l_b l_d dzeta,
            the coefficients of the homogeneous cubic of eq. (fIu2);
      Apoly, lag : the polynomials themselves.
    """
    alpha1 = Fraction(alpha1)
    c = tuple(Fraction(x) for x in c)
    nodes = (Fraction(0),) + c
    lag = lagrange_basis(nodes)
    Apoly = [A_poly_in_zeta(alpha1, ci) for ci in c]
    E = [[_pint01(_pmul(Apoly[i], lag[j])) for j in range(4)] for i in range(3)]
    C3 = [[[[None] * 4 for _ in range(4)] for _ in range(4)] for _ in range(3)]
    for i in range(3):
        for a in range(4):
            pa = _pmul(Apoly[i], lag[a])
            for b in range(4):
                pab = _pmul(pa, lag[b])
                for d in range(4):
                    C3[i][a][b][d] = _pint01(_pmul(pab, lag[d]))
    return {"alpha1": alpha1, "c": c, "nodes": nodes, "lag": lag, "Apoly": Apoly,
            "E": E, "C3": C3}


def constants_f64(alpha1=ALPHA1_PAPER, c=C_PAPER):
    """FP64 copies of E (3x4) and the cubic coefficient tensor (3x4x4x4)."""
    k = mb4_constants(Fraction(alpha1), tuple(Fraction(x) for x in c))
    E = np.array([[float(x) for x in row] for row in k["E"]], dtype=np.float64)
    C3 = np.array(k["C3"], dtype=object).astype(np.float64)
    return E, C3


# ---------------------------------------------------------------------------
# The discrete problem (Sec. 2.1).
# ---------------------------------------------------------------------------
def _circulant_adjacency(n):
    """C_n: periodic, zero diagonal, ones on the +-1 diagonals (D_n = C_n - 2 I)."""
    i = np.arange(n)
    rows = np.concatenate([i, i])
    cols = np.concatenate([(i + 1) % n, (i - 1) % n])
    data = np.ones(2 * n)
    return sp.csr_matrix((data, (rows, cols)), shape=(n, n))


def kinetic_matrix(nx, ny, tx, ty, eps0):
    """K = -tx (I_Ny (x) C_Nx) - ty (C_Ny (x) I_Nx) + eps0 I  (eq. Kdefinition,
    generalised).  Site k = y*Nx + x, so the x-direction operator sits in the
    right Kronecker factor."""
    if nx < 3 or ny < 3:
        raise ValueError("grid must be at least 3x3 so that the +-1 neighbours differ")
    Ix = sp.identity(nx, format="csr")
    Iy = sp.identity(ny, format="csr")
    K = (-tx * sp.kron(Iy, _circulant_adjacency(nx))
         - ty * sp.kron(_circulant_adjacency(ny), Ix)
         + eps0 * sp.identity(nx * ny))
    return sp.csr_matrix(K)


class Problem:
    """Grid, hopping, on-site shift, potential V (length S) and chi = -gamma:
    one value, or one per site -- the appendix's m-site model with a nonlinear
    energy U_I = -(1/2) sum_i gamma_i n_i^2, i.e. v_i = -gamma_i n_i."""

    def __init__(self, nx, ny, V, chi, tx=1.0, ty=None, eps0=0.0):
        self.nx, self.ny = int(nx), int(ny)
        self.S = self.nx * self.ny
        self.tx = float(tx)
        self.ty = float(tx if ty is None else ty)
        self.eps0 = float(eps0)
        self.V = np.asarray(V, dtype=np.float64).reshape(self.S).copy()
        self.chi = float(chi) if np.ndim(chi) == 0 else np.asarray(chi, dtype=np.float64).reshape(self.S).copy()
        self.K = kinetic_matrix(self.nx, self.ny, self.tx, self.ty, self.eps0)
        self.A = sp.csr_matrix(self.K + sp.diags(self.V))   # A = K + V (eq. JL)

    @classmethod
    def general(cls, K, V, chi):
        """A site model with a given kinetic matrix K (S x S, Hermitian, sparse or dense)
        instead of the grid stencil: the appendix's m-site model, in which K_kj is the
        transfer between neighbouring sites (complex, e.g. with Peierls phases; the
        paper asks only that K be Hermitian, Sec. 2.1 and the appendix).  A K with no
        imaginary part is kept real.  nx = S, ny = 1 label the sites."""
        K = sp.csr_matrix(K)
        if np.iscomplexobj(K.data) and not np.any(K.data.imag):
            K = sp.csr_matrix(K.real)
        K = sp.csr_matrix(K, dtype=np.complex128 if np.iscomplexobj(K.data) else np.float64)
        S = K.shape[0]
        if K.shape != (S, S) or (S and abs(K - K.conj().T).max() > 0):
            raise ValueError("K must be square and Hermitian")
        self = cls.__new__(cls)
        self.nx, self.ny, self.S = S, 1, S
        self.tx = self.ty = float("nan")
        self.eps0 = float("nan")
        self.V = np.asarray(V, dtype=np.float64).reshape(S).copy()
        self.chi = float(chi) if np.ndim(chi) == 0 else np.asarray(chi, dtype=np.float64).reshape(S).copy()
        self.K = K
        self.A = sp.csr_matrix(self.K + sp.diags(self.V))
        return self

    def f(self, u):
        """f(u) = f_K + f_I + f_E = -i[(K+V)u + chi |u|^2 u]  (eq. fdivide..fEu, gamma = -chi)."""
        return -1j * (self.A @ u + self.chi * (np.abs(u) ** 2) * u)


# ---------------------------------------------------------------------------
# Stage residual Phi(U), eq. (Phidefinition) with eq. (fKu2) and eq. (fIu2).
# ---------------------------------------------------------------------------
def residual(prob: Problem, u0, U, h, alpha1=ALPHA1_PAPER, c=C_PAPER):
    """Phi(U) for stages U (3, S) complex and step start u0 (S,) complex.

    Phi_i = U_i - u0 - h int_0^1 A_{c_i,zeta} f(U_zeta) dzeta, split as
      linear  : -i (K+V) (E_i0 u0 + sum_j E_ij U_j)               (eq. fKu2)
      cubic   : -i chi sum_{a,b,d} C3[i,a,b,d] conj(X_a) X_b X_d    (eq. fIu2)
    with X = (u0, U_1, U_2, U_3)."""
    E, C3 = constants_f64(alpha1, c)
    u0 = np.asarray(u0, dtype=np.complex128)
    U = np.asarray(U, dtype=np.complex128)
    X = np.vstack([u0[None, :], U])                         # (4, S)
    Y = E @ X                                                # (3, S): E_i0 u0 + sum_j E_ij U_j
    lin = -1j * np.vstack([prob.A @ Y[i] for i in range(3)])
    cub = -1j * prob.chi * np.einsum("iabd,ak,bk,dk->ik", C3, np.conj(X), X, X)
    return U - u0[None, :] - h * (lin + cub)


def residual_at_sites(nx, ny, V, chi, tx, ty, eps0, u0, U, h, sites,
                      alpha1=ALPHA1_PAPER, c=C_PAPER):
    """Phi(U) restricted to the listed sites (same formulas as ``residual``),
    touching only those sites and their four periodic neighbours, so that it
    can check a converged full-size stage vector one sample at a time."""
    E, C3 = constants_f64(alpha1, c)
    sites = np.asarray(sites, dtype=np.int64)
    u0 = np.asarray(u0, dtype=np.complex128)
    U = np.asarray(U, dtype=np.complex128)
    V = np.asarray(V, dtype=np.float64)
    y, x = np.divmod(sites, nx)
    xm, xp = (x - 1) % nx, (x + 1) % nx
    ym, yp = (y - 1) % ny, (y + 1) % ny
    nbx = [y * nx + xm, y * nx + xp]
    nby = [ym * nx + x, yp * nx + x]

    def Yat(idx):
        Xs = np.vstack([u0[idx][None, :], U[:, idx]])
        return E @ Xs

    Yc = Yat(sites)
    AY = ((eps0 + V[sites])[None, :] * Yc
          - tx * (Yat(nbx[0]) + Yat(nbx[1]))
          - ty * (Yat(nby[0]) + Yat(nby[1])))
    X = np.vstack([u0[sites][None, :], U[:, sites]])
    cub = np.einsum("iabd,ak,bk,dk->ik", C3, np.conj(X), X, X)
    chi_s = chi if np.ndim(chi) == 0 else np.asarray(chi, dtype=np.float64)[sites]
    return U[:, sites] - u0[sites][None, :] - h * (-1j) * (AY + chi_s * cub)


# ---------------------------------------------------------------------------
# Real form and the coupled simplified-Newton matrix.
# ---------------------------------------------------------------------------
def to_real(z):
    """Complex (..., S) -> real (..., 2S) as [p; q] (Sec. 2.1, real form)."""
    z = np.asarray(z)
    return np.concatenate([z.real, z.imag], axis=-1)


def to_complex(r, S):
    r = np.asarray(r)
    return r[..., :S] + 1j * r[..., S:]


def jacobian_real(prob: Problem, u0):
    """J = J_K + J_E + J_I at u0 in the real [p; q] form: eq. (JL) + eq. (JR)
    with gamma = -chi (per site when chi is):
      J_K + J_E = [[0, A], [-A, 0]]                 (A = K + V real),
      J_K + J_E = [[Im A, Re A], [-Re A, Im A]]     (A = K + V complex Hermitian: the
                  real form of -i A, whose real part acts as Re A q + Im A p and whose
                  imaginary part as -(Re A p - Im A q)),
      J_I = [[diag(-2 g p q), diag(-g (p^2 + 3 q^2))], [diag(g (3 p^2 + q^2)), diag(2 g p q)]]."""
    p0, q0 = np.real(u0), np.imag(u0)
    g = -prob.chi * np.ones_like(p0)
    A = prob.A
    if np.iscomplexobj(A.data):
        Ar, Ai = sp.csr_matrix(A.real), sp.csr_matrix(A.imag)
        JL = sp.bmat([[Ai, Ar], [-Ar, Ai]])
    else:
        JL = sp.bmat([[None, A], [-A, None]])
    JI = sp.bmat([[sp.diags(-2 * g * p0 * q0), sp.diags(-g * (p0 ** 2 + 3 * q0 ** 2))],
                  [sp.diags(g * (3 * p0 ** 2 + q0 ** 2)), sp.diags(2 * g * p0 * q0)]])
    return sp.csr_matrix(JL + JI)


def newton_matrix(prob: Problem, u0, h, alpha1=ALPHA1_PAPER, c=C_PAPER):
    """I_{3N} - h E (x) J  (eq. Jacobian2), N = 2S, coupled (not decoupled)."""
    E, _ = constants_f64(alpha1, c)
    J = jacobian_real(prob, u0)
    N = 2 * prob.S
    EJ = sp.kron(sp.csr_matrix(E[:, 1:]), J)
    return sp.csc_matrix(sp.identity(3 * N) - h * EJ)


class NewtonNotConverged(RuntimeError):
    pass


def _coupled_solver(M, method):
    """x = M^-1 rhs for the coupled Newton matrix: SuperLU, or scipy GMRES."""
    if method == "lu":
        lu = spla.splu(sp.csc_matrix(M))
        return lu.solve
    Mc = sp.csr_matrix(M)

    def solve(rhs):
        nrm = np.linalg.norm(rhs)
        if nrm == 0.0:
            return np.zeros_like(rhs)
        try:
            x, info = spla.gmres(Mc, rhs, rtol=1e-13, atol=0.0, restart=60, maxiter=50)
        except TypeError:   # older scipy spells the relative tolerance ``tol``
            x, info = spla.gmres(Mc, rhs, tol=1e-13, atol=0.0, restart=60, maxiter=50)
        if info != 0:
            raise RuntimeError(f"oracle GMRES did not converge (info={info})")
        return x
    return solve


def step(prob: Problem, u0, h, tol=1e-14, max_iter=50, alpha1=ALPHA1_PAPER, c=C_PAPER,
         return_stages=False, solver=None):
    """One MB4 step (Algorithm 1, one pass of its time loop) by simplified Newton
    on the coupled system (eq. Newton1).  Requires c3 = 1 so that u1 = U_c3.

    Stopping rule: ||r^l||_inf <= tol * ||u0||_inf (the paper's test on the
    update, made relative because the states here are normalised)."""
    if Fraction(c[2]) != 1:
        raise ValueError("the u1 = U_c3 shortcut needs c3 = 1")
    S = prob.S
    u0 = np.asarray(u0, dtype=np.complex128).reshape(S)
    if solver is None:
        solver = "lu" if S <= 1024 else "gmres"
    solve = _coupled_solver(newton_matrix(prob, u0, h, alpha1, c), solver)
    U = np.vstack([u0, u0, u0])                    # U^0 = e3 (x) u0
    scale = max(float(np.max(np.abs(np.concatenate([u0.real, u0.imag])))), 1e-300)
    for it in range(1, max_iter + 1):
        Phi = residual(prob, u0, U, h, alpha1, c)
        rhs = -np.concatenate([to_real(Phi[i]) for i in range(3)])
        r = solve(rhs)
        U = U + np.vstack([to_complex(r[i * 2 * S:(i + 1) * 2 * S], S) for i in range(3)])
        rho = float(np.max(np.abs(r)))
        if rho <= tol * scale:
            u1 = U[2].copy()
            return (u1, U, it) if return_stages else u1
    raise NewtonNotConverged(f"simplified Newton did not converge in {max_iter} iterations")


def run(prob: Problem, u0, h, nsteps, **kw):
    """nsteps MB4 steps from u0; returns the final state and the Newton counts."""
    u = np.asarray(u0, dtype=np.complex128).copy()
    counts = []
    for _ in range(nsteps):
        u, _, it = step(prob, u, h, return_stages=True, **kw)
        counts.append(it)
    return u, counts


# ---------------------------------------------------------------------------
# Observables (Sec. 2.1 energy terms; Sec. 3.2 participation ratio).
# ---------------------------------------------------------------------------
def energy(prob: Problem, u):
    """(H, U_K, U_E, U_nl) with U_K = u^H K u (real for Hermitian K), U_E = u^H V u,
    U_nl = (chi/2) sum |u|^4 = -(gamma/2) ||n||^2; correctly rounded sums."""
    u = np.asarray(u, dtype=np.complex128)
    Ku = prob.K @ u
    tK = np.real(np.conj(u) * Ku)
    n = np.abs(u) ** 2
    tE = prob.V * n
    tI = 0.5 * prob.chi * n * n
    UK = math.fsum(tK.tolist())
    UE = math.fsum(tE.tolist())
    UI = math.fsum(tI.tolist())
    H = math.fsum(np.concatenate([tK, tE, tI]).tolist())
    return H, UK, UE, UI


def norm2(u):
    return math.fsum((np.abs(np.asarray(u)) ** 2).tolist())


def participation(u):
    """p(t) = sum |u|^4 (Sec. 3.2, delta-potential experiment)."""
    return math.fsum((np.abs(np.asarray(u)) ** 4).tolist())
