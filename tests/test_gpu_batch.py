"""Batches of independent instances (mb4_batch_*): each instance gives the same
result alone and in the batch (up to the order of the Gram reductions, which
depends on the batch's grid), matches the oracle, and a failing or disabled
instance leaves the others untouched."""
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


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def _problems(nx, ny, B, seed0=0):
    V = np.stack([inputs.potential(nx, ny, 1.0, 3, 20.0, seed0 + b) for b in range(B)])
    chi = np.array([inputs.chi_for_seed(seed0 + b) for b in range(B)])
    chi[0] = 0.0                                  # one linear instance in every batch
    psi = np.stack([inputs.wavepacket(nx, ny, 2.5, math.pi / 4, 0.1 * b) for b in range(B)])
    return V, chi, psi


def _solo(mb4, nx, ny, V, chi, psi, h, steps, precision):
    with mb4.Integrator(nx, ny, V, chi, h, precision=precision) as it:
        it.set_state(psi)
        it.step(steps)
        return it.get_state()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_batch_matches_solo_runs(mb4, precision):
    nx, ny, B, h, steps = 24, 20, 5, 0.01, 10
    V, chi, psi = _problems(nx, ny, B)
    with mb4.Batch(nx, ny, V, chi, h, precision=precision) as bt:
        bt.set_state(psi)
        stats, codes = bt.step(steps)
        got = bt.get_state()
    assert codes == [0] * B
    assert all(s["steps_done"] == steps for s in stats)
    for b in range(B):
        want = _solo(mb4, nx, ny, V[b], chi[b], psi[b], h, steps, precision)
        assert _rel(got[b], want) <= 1e-12, (b, _rel(got[b], want))


def test_batch_matches_oracle(mb4):
    nx, ny, B, h, steps = 16, 16, 3, 0.01, 8
    V, chi, psi = _problems(nx, ny, B, seed0=11)
    with mb4.Batch(nx, ny, V, chi, h, precision="mixed") as bt:
        bt.set_state(psi)
        bt.step(steps)
        got = bt.get_state()
        obs = bt.observables()
    for b in range(B):
        prob = orc.Problem(nx, ny, V[b], chi[b])
        u, _ = orc.run(prob, psi[b], h, steps)
        assert _rel(got[b], u) <= 1e-11
        H = orc.energy(prob, u)[0]
        assert abs(obs[b, 0] - H) <= 1e-14 * abs(H)


def test_failing_instance_is_isolated(mb4):
    nx, ny, B, h, steps = 20, 20, 4, 0.01, 6
    V, chi, psi = _problems(nx, ny, B, seed0=3)
    bad = psi.copy()
    bad[2, 17] = np.nan
    with mb4.Batch(nx, ny, V, chi, h, precision="mixed") as bt:
        bt.set_state(bad)
        stats, codes = bt.step(steps)
        got = bt.get_state()
    assert codes[2] == mb4.MB4_ERR_NONFINITE
    assert stats[2]["steps_done"] == 0
    assert np.isnan(got[2, 17]) and np.array_equal(np.delete(got[2], 17), np.delete(bad[2], 17))
    for b in (0, 1, 3):
        assert codes[b] == 0
        want = _solo(mb4, nx, ny, V[b], chi[b], psi[b], h, steps, "mixed")
        assert _rel(got[b], want) <= 1e-12


def test_disable_and_load_slots(mb4):
    nx, ny, B, h = 16, 24, 3, 0.01
    V, chi, psi = _problems(nx, ny, B, seed0=7)
    with mb4.Batch(nx, ny, V, chi, h, precision="mixed") as bt:
        bt.set_state(psi)
        bt.enable(0, False)
        stats, codes = bt.step(4)
        assert stats[0]["steps_done"] == 0 and stats[1]["steps_done"] == 4
        assert np.array_equal(bt.get_state(0), psi[0])
        # reuse slot 2 for a new problem
        V2 = inputs.potential(nx, ny, 2.0, 5, 20.0, 99)
        psi2 = inputs.wavepacket(nx, ny, 3.0, 0.0, math.pi / 4)
        bt.load(2, V2, 1.5, psi2)
        bt.enable(0, True)
        stats, codes = bt.step(5)
        assert codes == [0, 0, 0]
        assert _rel(bt.get_state(2), _solo(mb4, nx, ny, V2, 1.5, psi2, h, 5, "mixed")) <= 1e-12
        assert _rel(bt.get_state(0), _solo(mb4, nx, ny, V[0], chi[0], psi[0], h, 5, "mixed")) <= 1e-12


def test_fp64_load_and_its_basis_scale_limit(mb4):
    """An FP64 batch scales its Krylov basis by tx: a reloaded slot gives its solo run,
    and a potential whose Gershgorin bound exceeds 4096 |tx| is refused (the mixed batch,
    scaled by that bound, takes it)."""
    nx, ny, B, h = 16, 24, 2, 0.01
    V, chi, psi = _problems(nx, ny, B, seed0=11)
    V2 = inputs.potential(nx, ny, 1.0, 4, 20.0, 123)
    psi2 = inputs.wavepacket(nx, ny, 2.0, math.pi / 4, 0.0)
    Vbig = V2.copy()
    Vbig[5] = 5000.0
    with mb4.Batch(nx, ny, V, chi, h, precision="fp64") as bt:
        bt.set_state(psi)
        bt.step(2)
        bt.load(1, V2, 0.7, psi2)
        stats, codes = bt.step(5)
        assert codes == [0, 0]
        assert _rel(bt.get_state(1), _solo(mb4, nx, ny, V2, 0.7, psi2, h, 5, "fp64")) <= 1e-12
        with pytest.raises(mb4.MB4Error) as e:
            bt.load(1, Vbig, 0.7, psi2)
        assert e.value.code == mb4.MB4_ERR_INVALID_ARG
    with mb4.Batch(nx, ny, V, chi, h, precision="mixed") as bt:
        bt.load(1, Vbig, 0.7, psi2)


def test_ensemble_1024_grid128_full_size(mb4):
    """The 1024-member 128x128 ensemble (chi ~ U[0, 2] per seed, 1% defects,
    sigma = 8, h = 0.01), mixed precision: two steps of the whole batch; sampled
    members match their own runs, conserve energy, and one matches the oracle."""
    B, n = 1024, 128
    ws = [inputs.ensemble128(seed) for seed in range(B)]
    V = np.stack([w.potential() for w in ws])
    chi = np.array([w.chi for w in ws])
    psi = np.stack([w.psi0() for w in ws])
    h = ws[0].h
    with mb4.Batch(n, n, V, chi, h, precision="mixed") as bt:
        bt.set_state(psi)
        obs0 = bt.observables()
        stats, codes = bt.step(2)
        got = bt.get_state()
        obs1 = bt.observables()
    assert codes == [0] * B
    drift = np.abs(obs1[:, 0] - obs0[:, 0]) / np.abs(obs0[:, 0])
    assert np.max(drift) <= 1e-13, np.max(drift)
    for b in (0, 1, 511, 1023):
        want = _solo(mb4, n, n, V[b], chi[b], psi[b], h, 2, "mixed")
        assert _rel(got[b], want) <= 1e-12
    prob = orc.Problem(n, n, V[5], chi[5])
    u, _ = orc.run(prob, psi[5], h, 2)
    assert _rel(got[5], u) <= 1e-11


@pytest.mark.parametrize("precision", PRECISIONS)
def test_batch_with_chi_field_and_preconditioner_matches_solo(mb4, precision):
    """Per-instance chi fields and the spectral preconditioner in a batch: each
    instance equals its own run."""
    nx, ny, B, h, steps = 24, 20, 3, 0.01, 6
    V, chi, psi = _problems(nx, ny, B, seed0=21)
    rng = np.random.default_rng(22)
    fields = rng.uniform(-2.0, 2.0, (B, nx * ny))
    with mb4.Batch(nx, ny, V, chi, h, precision=precision, site_chi=True, precondition=1) as bt:
        for b in range(B):
            bt.set_chi_field(b, fields[b])
        bt.set_state(psi)
        stats, codes = bt.step(steps)
        got = bt.get_state()
    assert codes == [0] * B
    for b in range(B):
        with mb4.Integrator(nx, ny, V[b], chi[b], h, precision=precision, site_chi=True, precondition=1) as it:
            it.set_chi_field(fields[b])
            it.set_state(psi[b])
            it.step(steps)
            assert _rel(got[b], it.get_state()) <= 1e-12
