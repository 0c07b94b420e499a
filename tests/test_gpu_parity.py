"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: GPU vs oracle <= 1e-11 relative in u after the stated steps, and
|dH/H| <= 1e-13 over a run, in both precision modes (FP32 inner solves do not
move the root of the stage equations).  The residual kernel on its own is
FP64 and must agree to rounding (1e-13 relative).
"""
import math

import numpy as np
import pytest

from oracle import mb4_oracle as orc
from paper_2003_04345_gb300 import inputs

pytestmark = pytest.mark.gpu

PRECISIONS = ["fp64", "mixed"]


@pytest.fixture(scope="module")
def mb4():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2003_04345_gb300 import mb4 as m
    m.lib()
    return m


def _rand_state(rng, S, scale=1.0):
    return scale * (rng.normal(size=S) + 1j * rng.normal(size=S))


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def _rel2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ---------------------------------------------------------------------------
# Residual kernel alone.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny", [(3, 3), (16, 16), (33, 17), (64, 40)])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_residual_kernel_matches_oracle(mb4, nx, ny, precision):
    rng = np.random.default_rng(nx * 100 + ny)
    S = nx * ny
    V = rng.uniform(-1, 1, S)
    V[rng.integers(0, S, 3)] += 20.0
    chi, tx, ty, eps0, h = 1.3, 1.1, 0.8, 0.25, 0.01
    prob = orc.Problem(nx, ny, V, chi, tx=tx, ty=ty, eps0=eps0)
    u0 = _rand_state(rng, S, 0.3)
    U = u0[None, :] + 0.05 * np.vstack([_rand_state(rng, S, 0.3) for _ in range(3)])
    want = orc.residual(prob, u0, U, h)
    with mb4.Integrator(nx, ny, V, chi, h, tx=tx, ty=ty, onsite=eps0, precision=precision) as it:
        got = it.residual(u0, U)
    scale = np.max(np.abs(U))
    assert np.max(np.abs(got - want)) <= 1e-13 * scale


# ---------------------------------------------------------------------------
# Shifted solves alone: (I - h lam_i J) x_i = b_i to the accuracy of one cycle.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision,s,eta", [("fp64", 10, 1e-7), ("fp64", 8, 1e-7), ("fp64", 5, 3e-5),
                                             ("mixed", 5, 3e-5), ("mixed", 8, 1e-5)])
def test_shifted_solves_reduce_residual(mb4, precision, s, eta):
    """One s-step GMRES cycle reduces ||b - (I - h lam_i J) x|| / ||b|| below eta
    for a random right-hand side on the 16x16 workload (h = 0.01), and lands within
    the matching distance of the dense LU solution of each shifted system."""
    w = inputs.grid16_fp64()
    S = w.S
    V = w.potential()
    rng = np.random.default_rng(3)
    u0 = w.psi0()
    b = np.vstack([_rand_state(rng, S) for _ in range(3)])
    prob = orc.Problem(w.nx, w.ny, V, w.chi, tx=w.tx, ty=w.ty, eps0=w.eps0)
    J = orc.jacobian_real(prob, u0)
    lam = mb4.constants()["lam"]
    with mb4.Integrator(w.nx, w.ny, V, w.chi, w.h, precision=precision, krylov_s=s) as it:
        x = it.solve_shifted(u0, b)
    for i in range(3):
        xr = orc.to_real(x[i])
        br = orc.to_real(b[i])
        res = br - (xr - w.h * lam[i] * (J @ xr))
        assert np.linalg.norm(res) <= eta * np.linalg.norm(br), (i, np.linalg.norm(res) / np.linalg.norm(br))
        A = np.eye(2 * S) - w.h * lam[i] * (J.toarray() if hasattr(J, "toarray") else J)
        xs = np.linalg.solve(A, br)                        # dense LU with partial pivoting
        bound = np.linalg.norm(np.linalg.inv(A), 2) * eta * np.linalg.norm(br)
        assert np.linalg.norm(xr - xs) <= 1.01 * bound, (i, np.linalg.norm(xr - xs), bound)


# ---------------------------------------------------------------------------
# Whole steps.
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def grid16_oracle_run():
    w = inputs.grid16_fp64()
    prob = orc.Problem(w.nx, w.ny, w.potential(), w.chi, tx=w.tx, ty=w.ty, eps0=w.eps0)
    u = w.psi0()
    H0 = orc.energy(prob, u)[0]
    traj = [u]
    for _ in range(w.steps):
        u = orc.step(prob, u, w.h)
        traj.append(u)
    return w, prob, traj, H0


@pytest.mark.parametrize("precision", PRECISIONS)
def test_grid16_trajectory_matches_oracle(mb4, grid16_oracle_run, precision):
    """16x16 wavepacket workload, 100 steps: <= 1e-11 relative in u at every 10th step."""
    w, prob, traj, H0 = grid16_oracle_run
    with mb4.from_workload(w, precision=precision) as it:
        drift = 0.0
        for n in range(10, w.steps + 1, 10):
            it.step(10)
            u = it.get_state()
            assert _rel(u, traj[n]) <= 1e-11, (n, _rel(u, traj[n]))
            assert _rel2(u, traj[n]) <= 1e-11
            H = it.energy()[0]
            drift = max(drift, abs(H - H0) / abs(H0))
        assert drift <= 1e-13, drift


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("order,adaptive", [(0, True), (1, True), (2, True), (3, True), (2, False), (3, False)])
def test_extrapolated_newton_start_matches_oracle(mb4, grid16_oracle_run, precision, order, adaptive):
    """Starting each step's Newton loop from extrapolated increments (order 0:
    Algorithm 1's U^0 = e3 (x) u0; adaptive: per step, the start that has recently
    been cheaper) moves only the start: the trajectory stays on the oracle's (1e-11)
    and conserves energy."""
    w, prob, traj, H0 = grid16_oracle_run
    with mb4.from_workload(w, precision=precision, newton_start=order, newton_start_adaptive=adaptive) as it:
        for n in range(20, w.steps + 1, 20):
            it.step(20)
            u = it.get_state()
            assert _rel(u, traj[n]) <= 1e-11, (n, _rel(u, traj[n]))
            assert abs(it.energy()[0] - H0) <= 1e-13 * abs(H0)


def test_set_state_forgets_the_newton_start_history_when_the_state_changes(mb4):
    w = inputs.grid16_fp64()
    with mb4.from_workload(w, newton_start=3) as a:
        a.step(6)
        new = a.get_state() * (1.0 + 1e-3)      # another state: the increments no longer fit
        a.set_state(new)
        a.step(5)
        ua = a.get_state()
    with mb4.Integrator(w.nx, w.ny, w.potential(), w.chi, w.h, newton_start=3) as b:
        b.set_state(new)
        b.step(5)
        assert np.array_equal(b.get_state(), ua)
    # writing back the very same state keeps the history (the host round trip of e2e use)
    with mb4.from_workload(w, newton_start=3) as c, mb4.from_workload(w, newton_start=3) as d:
        c.step(6)
        c.set_state(c.get_state())
        c.step(5)
        d.step(11)
        assert np.array_equal(c.get_state(), d.get_state())


@pytest.mark.parametrize("precision", PRECISIONS)
def test_stages_match_oracle(mb4, precision):
    rng = np.random.default_rng(21)
    nx, ny = 33, 17
    S = nx * ny
    V = rng.uniform(-0.5, 0.5, S)
    V[[5, 100, 400]] = 20.0
    prob = orc.Problem(nx, ny, V, 1.0)
    u0 = inputs.wavepacket(nx, ny, 3.0, math.pi / 4, 0.3)
    u1, U, _ = orc.step(prob, u0, 0.01, return_stages=True)
    with mb4.Integrator(nx, ny, V, 1.0, 0.01, precision=precision) as it:
        it.set_state(u0)
        it.step(1)
        Ug = it.stages()
        ug = it.get_state()
    assert _rel(Ug, U) <= 1e-12
    assert _rel(ug, u1) <= 1e-12
    assert np.array_equal(ug, Ug[2]) or _rel(ug, Ug[2]) <= 1e-15


@pytest.mark.parametrize("nx,ny", [(3, 3), (5, 7), (40, 24)])
def test_small_and_ragged_grids_match_oracle(mb4, nx, ny):
    rng = np.random.default_rng(nx + 7 * ny)
    S = nx * ny
    V = rng.uniform(-1, 1, S)
    chi, tx, ty, eps0, h = 0.8, 1.2, 0.7, 0.3, 0.02
    prob = orc.Problem(nx, ny, V, chi, tx=tx, ty=ty, eps0=eps0)
    u0 = _rand_state(rng, S, 0.5)
    u = u0
    for _ in range(5):
        u = orc.step(prob, u, h)
    for precision in PRECISIONS:
        with mb4.Integrator(nx, ny, V, chi, h, tx=tx, ty=ty, onsite=eps0, precision=precision) as it:
            it.set_state(u0)
            it.step(5)
            assert _rel(it.get_state(), u) <= 1e-11


@pytest.mark.parametrize("tx,ty", [(0.0, 0.8), (-0.7, 1.3), (0.002, 1.0)])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_stencil_forms_match_oracle(mb4, tx, ty, precision):
    """The three forms of the grid stencil: tx = 0 (the residual's plain stencil and the
    Gershgorin-scaled basis), tx < 0 (x hopping factored out, the FP64 basis scaled by a
    negative tx) and a tx so small that the FP64 basis keeps the Gershgorin scale while the
    residual still factors tx out."""
    nx, ny = 24, 20
    rng = np.random.default_rng(int(1000 * abs(tx)) + 31)
    S = nx * ny
    V = rng.uniform(-1, 1, S)
    V[rng.integers(0, S, 3)] += 20.0
    chi, eps0, h = 0.9, 0.2, 0.01
    prob = orc.Problem(nx, ny, V, chi, tx=tx, ty=ty, eps0=eps0)
    u0 = _rand_state(rng, S, 0.3)
    U = u0[None, :] + 0.05 * np.vstack([_rand_state(rng, S, 0.3) for _ in range(3)])
    u = u0
    for _ in range(5):
        u = orc.step(prob, u, h)
    with mb4.Integrator(nx, ny, V, chi, h, tx=tx, ty=ty, onsite=eps0, precision=precision) as it:
        got = it.residual(u0, U)
        assert np.max(np.abs(got - orc.residual(prob, u0, U, h))) <= 1e-13 * np.max(np.abs(U))
        it.set_state(u0)
        it.step(5)
        assert _rel(it.get_state(), u) <= 1e-11


def test_observables_match_oracle(mb4):
    rng = np.random.default_rng(8)
    nx, ny = 48, 20
    S = nx * ny
    V = rng.uniform(-1, 1, S)
    prob = orc.Problem(nx, ny, V, 1.7, tx=1.1, ty=0.9, eps0=0.2)
    u = _rand_state(rng, S, 0.1)
    with mb4.Integrator(nx, ny, V, 1.7, 0.01, tx=1.1, ty=0.9, onsite=0.2) as it:
        it.set_state(u)
        o = it.observables()
    H, UK, UE, UI = orc.energy(prob, u)
    for got, want in ((o["H"], H), (o["U_K"], UK), (o["U_E"], UE), (o["U_nl"], UI),
                      (o["norm2"], orc.norm2(u)), (o["participation"], orc.participation(u))):
        assert abs(got - want) <= 2e-15 * max(abs(want), 1e-300) + 1e-18, (got, want)


# ---------------------------------------------------------------------------
# Control flow, determinism, checkpoint/resume, failure detection.
# ---------------------------------------------------------------------------
def test_graph_and_host_loop_agree_bitwise(mb4):
    w = inputs.grid16_fp64()
    out = []
    for g in (True, False):
        with mb4.from_workload(w, use_graph=g) as it:
            st = it.step(10)
            out.append((it.get_state(), st["newton_iters_total"]))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("use_graph", [True, False])
def test_overlapped_launches_change_nothing(mb4, precision, use_graph):
    """Programmatic dependent launch only moves when blocks are scheduled: the
    results are bit for bit those of plain launches."""
    w = inputs.grid16_fp64()
    out = []
    for ov in (True, False):
        with mb4.from_workload(w, precision=precision, use_graph=use_graph, overlap_launches=ov) as it:
            st = it.step(12)
            out.append((it.get_state(), st["newton_iters_total"]))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


@pytest.mark.parametrize("precision", PRECISIONS)
def test_launch_shapes_change_nothing(mb4, precision):
    """Every threads-per-block choice the autotuner can make gives the same step bit
    for bit; the tuned shape is one of them."""
    w = inputs.grid16_fp64()
    out = []
    for bs in (64, 128, 256):
        with mb4.from_workload(w, precision=precision, site_threads=bs) as it:
            shape = it.launch_shape()
            assert shape[:4] == (bs,) * 4 and shape[4:] == ((w.S + bs - 1) // bs,) * 4
            it.step(8)
            out.append(it.get_state())
    assert all(np.array_equal(out[0], o) for o in out[1:])
    with mb4.from_workload(w, precision=precision, autotune=True) as it:
        shape = it.launch_shape()
        assert set(shape[:4]) <= {64, 128, 256} and all(g >= 1 for g in shape[4:])
        it.step(8)
        assert np.array_equal(it.get_state(), out[0])


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("start", [0, 2])
def test_deterministic_and_resumable(mb4, precision, start):
    """Runs repeat bit for bit.  Resuming from a saved state repeats them bit for bit
    with Algorithm 1's start; with the extrapolated start the resumed run has no
    history for its first steps, so it meets the same equations from another start
    and agrees to the Newton tolerance."""
    w = inputs.grid16_fp64()
    with mb4.from_workload(w, precision=precision, newton_start=start) as a:
        a.step(20)
        ua = a.get_state()
    with mb4.from_workload(w, precision=precision, newton_start=start) as b:
        b.step(20)
        ub = b.get_state()
    assert np.array_equal(ua, ub)
    with mb4.from_workload(w, precision=precision, newton_start=start) as c:
        c.step(10)
        mid = c.get_state()
    with mb4.Integrator(w.nx, w.ny, w.potential(), w.chi, w.h, precision=precision, newton_start=start) as d:
        d.set_state(mid)
        d.step(10)
        if start == 0:
            assert np.array_equal(d.get_state(), ua)
        else:
            assert _rel(d.get_state(), ua) <= 1e-13


@pytest.mark.parametrize("precision", PRECISIONS)
def test_async_steps_equal_synchronous_steps(mb4, precision):
    """mb4_step_async queues steps back to back; mb4_wait reports all of them."""
    w = inputs.grid16_fp64()
    with mb4.from_workload(w, precision=precision) as a:
        st_a = a.step(7)
        ua = a.get_state()
    with mb4.from_workload(w, precision=precision) as b:
        for n in (2, 3, 2):
            b.step_async(n)
        st_b = b.wait()
        assert np.array_equal(b.get_state(), ua)
        assert st_b["steps_done"] == 7 and st_b["newton_iters_total"] == st_a["newton_iters_total"]
        b.step_async(1)
        assert b.wait()["steps_done"] == 1          # counts restart at every wait


def test_pinned_host_buffers_equal_pageable_ones(mb4):
    """Page-locked host buffers are read and written in place by the pack and unpack
    kernels; pageable ones go through a staging copy.  Both give the same bits."""
    import torch
    w = inputs.grid16_fp64()
    psi = w.psi0()
    S = w.nx * w.ny
    hre = torch.from_numpy(np.ascontiguousarray(psi.real)).pin_memory()
    him = torch.from_numpy(np.ascontiguousarray(psi.imag)).pin_memory()
    outs = []
    for pinned in (False, True):
        with mb4.Integrator(w.nx, w.ny, w.potential(), w.chi, w.h, tx=w.tx, ty=w.ty, onsite=w.eps0) as it:
            if pinned:
                it.set_state_ptr(hre.data_ptr(), him.data_ptr(), 0)
            else:
                it.set_state(psi)
            it.step(3)
            if pinned:
                a = torch.empty(S, dtype=torch.float64).pin_memory()
                b = torch.empty(S, dtype=torch.float64).pin_memory()
                it.get_state_ptr(a.data_ptr(), b.data_ptr(), 0)
                outs.append(a.numpy() + 1j * b.numpy())
                assert np.array_equal(outs[-1], it.get_state())
            else:
                outs.append(it.get_state())
    assert np.array_equal(outs[0], outs[1])


def test_async_failure_is_reported_by_wait(mb4):
    w = inputs.grid16_fp64()
    with mb4.from_workload(w, newton_max=1) as it:
        u0 = it.get_state()
        it.step_async(2)
        it.step_async(2)
        st, rc = it.wait(check=False)
        assert rc == mb4.MB4_ERR_NEWTON_NOT_CONVERGED and st["steps_done"] == 0
        assert np.array_equal(it.get_state(), u0)


def test_time_reversal_on_gpu(mb4):
    w = inputs.grid16_fp64()
    V = w.potential()
    with mb4.from_workload(w) as f, mb4.Integrator(w.nx, w.ny, V, w.chi, -w.h) as b:
        u0 = f.get_state()
        f.step(5)
        b.set_state(f.get_state())
        b.step(5)
        assert _rel(b.get_state(), u0) <= 1e-13


def test_newton_failure_keeps_last_state(mb4):
    w = inputs.grid16_fp64()
    with mb4.from_workload(w, newton_max=1) as it:
        u0 = it.get_state()
        st, rc = it.step(3, check=False)
        assert rc == mb4.MB4_ERR_NEWTON_NOT_CONVERGED
        assert st["steps_done"] == 0
        assert np.array_equal(it.get_state(), u0)


def test_nonfinite_state_is_reported(mb4):
    w = inputs.grid16_fp64()
    with mb4.from_workload(w) as it:
        psi = w.psi0()
        psi[17] = np.nan
        it.set_state(psi)
        st, rc = it.step(2, check=False)
        assert rc == mb4.MB4_ERR_NONFINITE
        assert st["steps_done"] == 0
        after = it.get_state()
        assert np.isnan(after[17]) and np.array_equal(np.delete(after, 17), np.delete(psi, 17))


@pytest.mark.parametrize("precision", PRECISIONS)
def test_chi_field_matches_oracle(mb4, precision):
    """Per-site chi (the appendix's m-site model, both signs) through set_chi_field:
    the trajectory stays on the oracle's, the observables equal the oracle's energy
    of the GPU state, and the field model's energy is conserved."""
    nx, ny, h, steps = 24, 20, 0.01, 10
    rng = np.random.default_rng(41)
    V = inputs.potential(nx, ny, 1.0, 3, 20.0, 5)
    chi = rng.uniform(-2.0, 2.0, nx * ny)
    psi = inputs.wavepacket(nx, ny, 2.5, math.pi / 4, 0.0)
    prob = orc.Problem(nx, ny, V, chi)
    u = psi.copy()
    for _ in range(steps):
        u = orc.step(prob, u, h)
    with mb4.Integrator(nx, ny, V, 0.0, h, precision=precision, site_chi=True) as it:
        it.set_chi_field(chi)
        it.set_state(psi)
        H0 = it.energy()[0]
        assert abs(H0 - orc.energy(prob, psi)[0]) <= 1e-14 * abs(H0)
        it.step(steps)
        got = it.get_state()
        assert _rel(got, u) <= 1e-11, _rel(got, u)
        H1 = it.energy()[0]
        assert abs(H1 - orc.energy(prob, got)[0]) <= 1e-14 * abs(H1)
        assert abs(H1 - H0) <= 1e-13 * abs(H0)
    with mb4.Integrator(nx, ny, V, 1.0, h) as it:
        with pytest.raises(mb4.MB4Error):
            it.set_chi_field(chi)                        # the context has no field


def test_uniform_chi_field_equals_scalar_chi(mb4):
    w = inputs.grid16_fp64()
    with mb4.from_workload(w) as a, mb4.from_workload(w, site_chi=True) as b:
        a.step(10)
        b.step(10)                                       # field initialised to the scalar chi
        assert _rel(b.get_state(), a.get_state()) <= 1e-13


@pytest.mark.parametrize("precision", PRECISIONS)
def test_degenerate_inputs(mb4, precision):
    """Zero steps leave everything as it was; the zero state is a fixed point (its
    residual is exactly 0, so one Newton iteration confirms it); a single-site-wide
    ragged grid and a negative h run like any other."""
    w = inputs.grid16_fp64()
    with mb4.from_workload(w, precision=precision) as it:
        u0 = it.get_state()
        st = it.step(0)
        assert st["steps_done"] == 0 and np.array_equal(it.get_state(), u0)
        it.set_state(np.zeros(w.S, dtype=np.complex128))
        st = it.step(3)
        assert st["steps_done"] == 3 and not np.any(it.get_state())
        assert it.energy()[0] == 0.0
    nx, ny = 3, 41                                        # 3 x 41 periodic strip
    rng = np.random.default_rng(61)
    V = rng.uniform(-1, 1, nx * ny)
    psi = rng.normal(size=nx * ny) + 1j * rng.normal(size=nx * ny)
    prob = orc.Problem(nx, ny, V, 0.8, tx=0.9, ty=1.1, eps0=0.1)
    u = psi.copy()
    for _ in range(4):
        u = orc.step(prob, u, -0.01)
    with mb4.Integrator(nx, ny, V, 0.8, -0.01, tx=0.9, ty=1.1, onsite=0.1, precision=precision) as it:
        it.set_state(psi)
        it.step(4)
        assert _rel(it.get_state(), u) <= 1e-11


def test_invalid_arguments_rejected(mb4):
    for kw in ({"nx": 2, "ny": 8}, {"h": 0.0}, {"krylov_s": 11}, {"precision": 7}, {"site_threads": 96},
               {"newton_start": 4}):
        args = {"nx": 4, "ny": 4, "h": 0.01}
        args.update(kw)
        nx, ny = args.pop("nx"), args.pop("ny")
        with pytest.raises((mb4.MB4Error, ValueError, KeyError)):
            mb4.Integrator(nx, ny, np.zeros(nx * ny), 1.0, **args)


# ---------------------------------------------------------------------------
# Full size (the benchmark's configuration): checks the oracle can make one site
# at a time, and properties that hold at any size.
# ---------------------------------------------------------------------------
def _sample_sites(w, n, seed):
    rng = np.random.default_rng(seed)
    edges = [0, w.nx - 1, w.S - w.nx, w.S - 1, w.nx * (w.ny // 2)]
    V = w.potential()
    defects = list(np.nonzero(V > 10)[0][:8])
    return np.unique(np.concatenate([edges, defects, rng.integers(0, w.S, n)]))


@pytest.mark.parametrize("precision", PRECISIONS)
def test_grid512_stages_solve_oracle_stage_equations(mb4, precision):
    """512x512, bench configuration: after each of 3 steps the converged stages
    satisfy the oracle's Phi(U) = 0 at sampled sites to the Newton tolerance."""
    w = inputs.grid512_fp64()
    V = w.potential()
    with mb4.from_workload(w, precision=precision) as it:
        u0 = it.get_state()
        H0 = it.energy()[0]
        for n in range(3):
            st = it.step(1)
            U = it.stages()
            sites = _sample_sites(w, 300, n)
            phi = orc.residual_at_sites(w.nx, w.ny, V, w.chi, w.tx, w.ty, w.eps0, u0, U, w.h, sites)
            assert np.max(np.abs(phi)) <= 1e-13 * np.max(np.abs(u0)), np.max(np.abs(phi))
            u0 = it.get_state()
            assert np.array_equal(u0, U[2]) or _rel(u0, U[2]) < 1e-15
        H = it.energy()[0]
        assert abs(H - H0) <= 1e-13 * abs(H0)


def test_grid512_translation_equivariance(mb4):
    w = inputs.grid512_fp64()
    V = w.potential().reshape(w.ny, w.nx)
    psi = w.psi0().reshape(w.ny, w.nx)
    roll = lambda a: np.roll(np.roll(a, 37, axis=1), -101, axis=0)
    with mb4.Integrator(w.nx, w.ny, V.ravel(), w.chi, w.h) as a, \
            mb4.Integrator(w.nx, w.ny, roll(V).ravel(), w.chi, w.h) as b:
        a.set_state(psi.ravel())
        b.set_state(roll(psi).ravel())
        a.step(3)
        b.step(3)
        ua = a.get_state().reshape(w.ny, w.nx)
        ub = b.get_state().reshape(w.ny, w.nx)
    assert _rel(ub, roll(ua)) <= 1e-13


def test_grid2048_mixed_matches_fp64(mb4):
    """2048x2048 (W = 2, 1% defects, chi = 2, h = 0.002): FP32 inner solves do not
    move the root -- mixed and FP64 agree to the parity tolerance after 3 steps, and in
    both the third step's stages satisfy the oracle's Phi(U) = 0 at sampled sites."""
    w = inputs.grid2048_mixed()
    V = w.potential()
    finals = {}
    for precision in PRECISIONS:
        with mb4.from_workload(w, precision=precision) as it:
            H0 = it.energy()[0]
            it.step(2)
            u0 = it.get_state()
            it.step(1)
            U = it.stages()
            sites = _sample_sites(w, 300, 7)
            phi = orc.residual_at_sites(w.nx, w.ny, V, w.chi, w.tx, w.ty, w.eps0, u0, U, w.h, sites)
            assert np.max(np.abs(phi)) <= 1e-13 * np.max(np.abs(u0)), np.max(np.abs(phi))
            finals[precision] = it.get_state()
            assert abs(it.energy()[0] - H0) <= 1e-13 * abs(H0)
    assert _rel(finals["mixed"], finals["fp64"]) <= 1e-11


@pytest.mark.oracle_long("c3_crop")
@pytest.mark.parametrize("precision", PRECISIONS)
def test_grid128_with_2048_physics_matches_oracle(mb4, precision):
    """The 128x128 instance with the 2048x2048 physics over its whole 500 steps against
    the oracle (the error of the 2048x2048 configuration stated at the size the oracle can
    follow): 1e-11 relative in l-inf and l2 after 10, 100, 250 and 500 steps, and the
    GPU's energy within 1e-13 of the oracle's start every 10 steps."""
    import oracle_jobs
    w = inputs.grid128_crop_of_2048()
    want = oracle_jobs.result("c3_crop")
    errs = {}
    with mb4.from_workload(w, precision=precision) as it:
        H0 = it.energy()[0]
        assert abs(H0 - want["H"][0]) <= 1e-14 * abs(want["H"][0])
        for n in range(1, w.steps // 10 + 1):
            it.step(10)
            H = it.energy()[0]
            assert abs(H - want["H"][0]) <= 1e-13 * abs(want["H"][0]), (10 * n, H)
            if 10 * n in want:
                got = it.get_state()
                errs[10 * n] = (_rel(got, want[10 * n]), _rel2(got, want[10 * n]))
    assert sorted(errs) == [10, 100, 250, 500]
    print(f"\n[{precision}] 128x128 with the 2048x2048 physics vs the oracle, step: (rel l-inf, rel l2) "
          + ", ".join(f"{n}: ({a:.2e}, {b:.2e})" for n, (a, b) in sorted(errs.items())))
    for n, (einf, e2) in errs.items():
        assert einf <= 1e-11 and e2 <= 1e-11, (n, einf, e2)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_energy_drift_long_run(mb4, precision):
    """4000 steps (64x64, h = 0.01, 2% defects, chi = 1): |dH/H| stays at the
    1e-13 level with no drift proportional to the step count (a systematic
    per-step bias of 1e-16 would reach 4e-13 here)."""
    w = inputs.Workload("long64", 64, 64, h=0.01, steps=4000, chi=1.0, W=1.0, defect_fraction=0.02,
                        sigma=6.0, seed=17)
    with mb4.from_workload(w, precision=precision, newton_predict=1e-16) as it:
        H0 = it.energy()[0]
        worst = 0.0
        for _ in range(8):
            it.step(w.steps // 8)
            worst = max(worst, abs(it.energy()[0] - H0) / abs(H0))
    assert worst <= 1e-13, worst


def _random_graph(S, deg, seed, onsite=0.3):
    rng = np.random.default_rng(seed)
    K = np.zeros((S, S))
    for k in range(S):
        for j in rng.choice(S, size=deg // 2, replace=False):
            if j != k:
                K[k, j] = K[j, k] = rng.uniform(-1.5, 1.5)
    return K + onsite * np.eye(S)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_general_kinetic_matrix_matches_oracle(mb4, precision):
    """A general sparse K (mb4_create_sparse; the appendix's m-site model on a random
    graph, with a per-site chi): trajectory and energy against the oracle."""
    S, h, steps = 300, 0.01, 10
    K = _random_graph(S, 6, 51)
    rng = np.random.default_rng(52)
    V = rng.uniform(-1, 1, S)
    chi = rng.uniform(-2, 2, S)
    psi = (rng.normal(size=S) + 1j * rng.normal(size=S)) / np.sqrt(2 * S)
    prob = orc.Problem.general(K, V, chi)
    u = psi.copy()
    for _ in range(steps):
        u = orc.step(prob, u, h)
    with mb4.Integrator.sparse(K, V, 0.0, h, precision=precision, site_chi=True) as it:
        it.set_chi_field(chi)
        it.set_state(psi)
        H0 = it.energy()[0]
        assert abs(H0 - orc.energy(prob, psi)[0]) <= 1e-14 * abs(H0)
        it.step(steps)
        got = it.get_state()
        assert _rel(got, u) <= 1e-11, _rel(got, u)
        assert abs(it.energy()[0] - H0) <= 1e-13 * abs(H0)


def _random_hermitian_graph(S, deg, seed, onsite=0.3):
    """Random sparse Hermitian K: links t e^{i phi} (Peierls-like phases)."""
    rng = np.random.default_rng(seed)
    K = np.zeros((S, S), dtype=np.complex128)
    for k in range(S):
        for j in rng.choice(S, size=deg // 2, replace=False):
            if j != k:
                w = rng.uniform(-1.5, 1.5) * np.exp(1j * rng.uniform(-math.pi, math.pi))
                K[k, j] = w
                K[j, k] = np.conj(w)
    return K + onsite * np.eye(S)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_complex_hermitian_kinetic_matrix_matches_oracle(mb4, precision):
    """A complex Hermitian K (the m-site model with Peierls-like phases on a random graph,
    per-site chi): trajectory to 1e-11 and energy to 1e-13 against the oracle."""
    S, h, steps = 300, 0.01, 10
    K = _random_hermitian_graph(S, 6, 61)
    rng = np.random.default_rng(62)
    V = rng.uniform(-1, 1, S)
    chi = rng.uniform(-2, 2, S)
    psi = (rng.normal(size=S) + 1j * rng.normal(size=S)) / np.sqrt(2 * S)
    prob = orc.Problem.general(K, V, chi)
    u = psi.copy()
    for _ in range(steps):
        u = orc.step(prob, u, h)
    with mb4.Integrator.sparse(K, V, 0.0, h, precision=precision, site_chi=True) as it:
        it.set_chi_field(chi)
        it.set_state(psi)
        H0 = it.energy()[0]
        assert abs(H0 - orc.energy(prob, psi)[0]) <= 1e-14 * abs(H0)
        o = it.observables()
        _, UK, UE, UI = orc.energy(prob, psi)
        for got, want in ((o["U_K"], UK), (o["U_E"], UE), (o["U_nl"], UI)):
            assert abs(got - want) <= 1e-14 * (abs(UK) + abs(UE) + abs(UI))
        it.step(steps)
        got = it.get_state()
        assert _rel(got, u) <= 1e-11, _rel(got, u)
        assert _rel2(got, u) <= 1e-11
        assert abs(it.energy()[0] - H0) <= 1e-13 * abs(H0)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_gauge_transformed_grid_equals_the_grid(mb4, precision):
    """K' = G K G^H with G = diag(e^{i theta}) and K the 5-point stencil: the complex
    sparse path started from G u0 gives G times the grid path's result (a symmetry of
    the equation that MB4 keeps), to 1e-13 after 10 steps."""
    w = inputs.grid16_fp64()
    prob = orc.Problem(w.nx, w.ny, w.potential(), w.chi, tx=w.tx, ty=w.ty, eps0=w.eps0)
    theta = np.random.default_rng(63).uniform(-math.pi, math.pi, w.S)
    G = np.exp(1j * theta)
    Kc = (G[:, None] * prob.K.toarray()) * np.conj(G)[None, :]
    Kc = 0.5 * (Kc + Kc.conj().T)
    with mb4.from_workload(w, precision=precision) as a, \
            mb4.Integrator.sparse(Kc, w.potential(), w.chi, w.h, precision=precision) as b:
        b.set_state(G * w.psi0())
        a.step(10)
        b.step(10)
        assert _rel(b.get_state(), G * a.get_state()) <= 1e-13


def test_complex_kinetic_matrix_rejects_a_non_hermitian_one(mb4):
    from paper_2003_04345_gb300.mb4 import C, Nonlinearity, Potential, SparseKinetic, _P, _options, lib
    S = 4
    V = np.zeros(S)
    nb = np.ascontiguousarray(np.array([[1], [0], [3], [2]], dtype=np.int32))
    tt = np.ascontiguousarray(np.ones((4, 1)))
    for ti in ([[0.5], [0.5], [0.2], [-0.2]],      # Im K_01 = Im K_10: symmetric, not Hermitian
               [[0.5], [-0.4], [0.0], [0.0]]):     # not the conjugate
        tim = np.ascontiguousarray(np.array(ti, dtype=np.float64))
        ctx = _P()
        rc = lib().mb4_create_sparse(C.byref(SparseKinetic(S, 1, nb.ctypes.data, tt.ctypes.data, 0.0,
                                                           tim.ctypes.data)),
                                     C.byref(Potential(V.ctypes.data, 0)), C.byref(Nonlinearity(1.0)), 0.01,
                                     C.byref(_options()), C.byref(ctx))
        assert rc == mb4.MB4_ERR_INVALID_ARG
    tim = np.ascontiguousarray(np.array([[0.5], [-0.5], [0.2], [-0.2]], dtype=np.float64))
    ctx = _P()
    rc = lib().mb4_create_sparse(C.byref(SparseKinetic(S, 1, nb.ctypes.data, tt.ctypes.data, 0.0, tim.ctypes.data)),
                                 C.byref(Potential(V.ctypes.data, 0)), C.byref(Nonlinearity(1.0)), 0.01,
                                 C.byref(_options()), C.byref(ctx))
    assert rc == mb4.MB4_OK
    lib().mb4_destroy(ctx)


def test_general_kinetic_matrix_of_the_grid_equals_the_grid(mb4):
    """The 5-point stencil handed over as a matrix gives the grid context's step."""
    w = inputs.grid16_fp64()
    prob = orc.Problem(w.nx, w.ny, w.potential(), w.chi, tx=w.tx, ty=w.ty, eps0=w.eps0)
    with mb4.from_workload(w) as a, mb4.Integrator.sparse(prob.K, w.potential(), w.chi, w.h) as b:
        b.set_state(w.psi0())
        a.step(10)
        b.step(10)
        assert _rel(b.get_state(), a.get_state()) <= 1e-13


def test_general_kinetic_matrix_rejects_bad_input(mb4):
    from paper_2003_04345_gb300.mb4 import C, Nonlinearity, Potential, SparseKinetic, _P, _options, lib
    S = 4
    V = np.zeros(S)
    for nbr, t in (([[1], [0], [3], [2]], [[1.0], [2.0], [1.0], [1.0]]),      # not symmetric
                   ([[0], [0], [3], [2]], [[1.0], [1.0], [1.0], [1.0]]),      # a self link
                   ([[5], [0], [3], [2]], [[1.0], [1.0], [1.0], [1.0]])):     # out of range
        nb = np.ascontiguousarray(np.array(nbr, dtype=np.int32))
        tt = np.ascontiguousarray(np.array(t, dtype=np.float64))
        ctx = _P()
        rc = lib().mb4_create_sparse(C.byref(SparseKinetic(S, 1, nb.ctypes.data, tt.ctypes.data, 0.0)),
                                     C.byref(Potential(V.ctypes.data, 0)), C.byref(Nonlinearity(1.0)), 0.01,
                                     C.byref(_options()), C.byref(ctx))
        assert rc == mb4.MB4_ERR_INVALID_ARG and not ctx.value


@pytest.mark.parametrize("tile", list(range(1, 16)))
def test_matrix_powers_tiles_give_the_same_steps(mb4, tile):
    """Every form of the FP32 Krylov basis the tuner chooses among (the matrix-powers tiles,
    and one stencil launch per level) builds the same basis bit for bit, so the mixed step
    is the same: a grid whose sides are not multiples of any tile (ragged tiles at both
    edges)."""
    w = inputs.Workload("ragged", 100, 70, h=0.005, steps=10, chi=1.0, W=1.0, defect_fraction=0.01, sigma=5.0)
    with mb4.from_workload(w, precision="mixed", powers_tile=tile) as it:
        assert it.tile_shape() == [(32, 16), (32, 32), (64, 16), (32, 8), (32, 16), (64, 16), (32, 16), (64, 16),
                                   (24, 4), (24, 8), (24, 8), (24, 16), (24, 8), (24, 16), (0, 0)][tile - 1]
        it.step(10)
        got = it.get_state()
    with mb4.from_workload(w, precision="mixed", powers_tile=1) as it:
        it.step(10)
        want = it.get_state()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("s", [2, 3, 5, 6])
@pytest.mark.parametrize("tile", [9, 10, 11, 12, 13, 14, 15])
def test_warp_and_level_forms_other_s_and_small_grids(mb4, s, tile):
    """The one-warp tiles and strips (interior 32 - 2s wide) and the per-level launches at
    every other s they take, on a grid narrower than one warp tile (17 x 13: the tile wraps
    onto itself, and a strip is taller than the grid) and on a ragged one: the same steps
    as the 32 x 16 tile."""
    for nx, ny in ((17, 13), (61, 45)):
        w = inputs.Workload("small", nx, ny, h=0.005, steps=6, chi=1.0, W=1.0, defect_fraction=0.02, sigma=3.0)
        out = []
        for t in (tile, 1):
            with mb4.from_workload(w, precision="mixed", krylov_s=s, powers_tile=t) as it:
                it.step(6)
                out.append(it.get_state())
        assert np.array_equal(out[0], out[1]), (nx, ny)
