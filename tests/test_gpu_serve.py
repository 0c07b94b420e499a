"""Continuous-batching server (mb4_server_*): requests of different grid sizes,
step sizes, step counts and potentials arrive over time, share the GPU inside an
HBM budget, and each result equals the same simulation run alone."""
import math

import numpy as np
import pytest

from paper_2003_04345_gb300 import inputs

pytestmark = pytest.mark.gpu


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


def _trace(n_req, seed=0, span=0.05):
    rng = np.random.default_rng(seed)
    sizes = [(16, 16), (24, 24), (32, 20)]
    hs = [0.01, 0.005]
    reqs = []
    for r in range(n_req):
        nx, ny = sizes[rng.integers(len(sizes))]
        h = hs[rng.integers(len(hs))]
        steps = int(rng.integers(3, 41))
        chi = float(rng.uniform(0, 2))
        V = inputs.potential(nx, ny, 1.0, 2, 20.0, 100 + r)
        psi = inputs.wavepacket(nx, ny, 2.5, math.pi / 4, 0.2 * (r % 3))
        reqs.append(dict(nx=nx, ny=ny, h=h, nsteps=steps, chi=chi, V=V, psi=psi, arrival=float(span * r / n_req)))
    return reqs


def _solo(mb4, q, **opts):
    with mb4.Integrator(q["nx"], q["ny"], q["V"], q["chi"], q["h"], **opts) as it:
        it.set_state(q["psi"])
        it.step(q["nsteps"])
        return it.get_state()


def _oracle(q):
    from oracle import mb4_oracle as orc
    prob = orc.Problem(q["nx"], q["ny"], q["V"], q["chi"])
    u = q["psi"].copy()
    for _ in range(q["nsteps"]):
        u = orc.step(prob, u, q["h"])
    return u


def test_served_results_equal_solo_runs(mb4):
    """A burst of 14 requests over 6 shape classes with 2 slots per batch: the
    classes run concurrently, every result equals its solo run, and every result
    matches the FP64 oracle's run of the same request to 1e-11 (so the served path is
    pinned to the oracle directly, not only through the solo path)."""
    reqs = _trace(14, span=0.0)
    with mb4.Server(2 << 30, max_slots=2, keep_states=True, precision="mixed") as srv:
        ids = [srv.submit(q["nx"], q["ny"], q["V"], q["chi"], q["psi"], q["h"], q["nsteps"], q["arrival"])
               for q in reqs]
        done = srv.run()
        assert done == len(reqs)
        results = [srv.result(i, state=True) for i in ids]
    spans = []
    for q, (res, u) in zip(reqs, results):
        assert res["done"] == 1 and res["status"] == 0
        assert res["steps_done"] == q["nsteps"]
        assert res["admitted"] >= res["arrival"] - 1e-9 and res["completed"] >= res["admitted"]
        assert abs(res["energy_end"] - res["energy_start"]) <= 1e-13 * abs(res["energy_start"])
        assert _rel(u, _solo(mb4, q, precision="mixed")) <= 1e-12
        assert _rel(u, _oracle(q)) <= 1e-11
        spans.append((res["admitted"], res["completed"], (q["nx"], q["ny"], q["h"])))
    # different requests were on the GPU at the same time
    overlaps = sum(1 for i in range(len(spans)) for j in range(i + 1, len(spans))
                   if spans[i][0] < spans[j][1] and spans[j][0] < spans[i][1])
    assert overlaps > 0


def test_waiting_requests_take_freed_slots(mb4):
    """One shape class, five requests, a budget that holds a single two-slot batch:
    two requests run together, and the others are admitted into the slots the
    finished ones free (continuous batching within the memory budget)."""
    reqs = _trace(5, seed=2, span=0.0)
    for r, q in enumerate(reqs):
        q.update(nx=32, ny=20, h=0.01, nsteps=10 + 7 * r)
        q["V"] = inputs.potential(32, 20, 1.0, 2, 20.0, 50 + r)
        q["psi"] = inputs.wavepacket(32, 20, 2.5, math.pi / 4, 0.1 * r)
    two = mb4.batch_bytes(32, 20, 2, precision="mixed")
    with mb4.Server(two + two // 4, max_slots=2, keep_states=True, precision="mixed") as srv:
        ids = [srv.submit(q["nx"], q["ny"], q["V"], q["chi"], q["psi"], q["h"], q["nsteps"], 0.0) for q in reqs]
        assert srv.run() == len(reqs)
        results = [srv.result(i, state=True) for i in ids]
    spans = []
    for q, (res, u) in zip(reqs, results):
        assert res["status"] == 0 and res["steps_done"] == q["nsteps"]
        assert _rel(u, _solo(mb4, q, precision="mixed")) <= 1e-12
        assert _rel(u, _oracle(q)) <= 1e-11
        spans.append((res["admitted"], res["completed"]))
    assert any(a[0] < b[1] and b[0] < a[1] for a in spans for b in spans if a is not b)   # ran together
    assert sum(1 for b in spans if any(b[0] >= a[1] for a in spans if a is not b)) >= 3  # waited for a slot


def test_small_request_finishes_while_a_large_class_is_mid_chunk(mb4):
    """Each shape class is polled on its own: a 1024 x 1024 request of 256 steps (8 chunks
    of 32 steps) arrives first, a 32 x 32 request of 20 steps 5 ms later.  The small one is
    admitted, stepped and retired while the large class is inside one of its chunks: its
    latency is well under one large chunk, instead of waiting for the large chunk to end."""
    big = dict(nx=1024, ny=1024, h=0.002, nsteps=256, chi=1.0, arrival=0.0,
               V=inputs.potential(1024, 1024, 1.0, 10000, 20.0, 11),
               psi=inputs.wavepacket(1024, 1024, 16.0, math.pi / 4, 0.0))
    small = dict(nx=32, ny=32, h=0.01, nsteps=20, chi=1.0, arrival=0.005,
                 V=inputs.potential(32, 32, 1.0, 10, 20.0, 12),
                 psi=inputs.wavepacket(32, 32, 3.0, math.pi / 4, 0.0))
    with mb4.Server(8 << 30, max_slots=2, keep_states=True, precision="mixed") as srv:
        ids = [srv.submit(q["nx"], q["ny"], q["V"], q["chi"], q["psi"], q["h"], q["nsteps"], q["arrival"])
               for q in (big, small)]
        assert srv.run() == 2
        (rb, _), (rs, us) = [srv.result(i, state=True) for i in ids]
    assert rb["status"] == 0 and rs["status"] == 0
    chunk = (rb["completed"] - rb["admitted"]) / 8
    assert rs["completed"] < rb["completed"]
    # stepped and retired within half a large chunk of its admission (which came as soon as
    # its own class batch existed: the large class's chunk did not hold it back)
    assert rs["completed"] - rs["admitted"] < 0.5 * chunk, (rs["completed"] - rs["admitted"], chunk)
    assert rs["admitted"] - rs["arrival"] < 2 * chunk, (rs["admitted"] - rs["arrival"], chunk)
    assert _rel(us, _oracle(small)) <= 1e-11


def test_budget_limits_concurrency(mb4):
    reqs = [dict(q, nx=32, ny=20) for q in _trace(5, seed=1)]
    for q in reqs:
        q["V"] = inputs.potential(32, 20, 1.0, 2, 20.0, 7)
        q["psi"] = inputs.wavepacket(32, 20, 2.5, math.pi / 4, 0.0)
    one = mb4.batch_bytes(32, 20, 1, precision="mixed")
    with mb4.Server(one + one // 2, max_slots=8, keep_states=True, precision="mixed") as srv:
        ids = [srv.submit(q["nx"], q["ny"], q["V"], q["chi"], q["psi"], q["h"], q["nsteps"], 0.0) for q in reqs]
        assert srv.run() == len(reqs)
        results = [srv.result(i, state=True) for i in ids]
    by_h = {}
    for q, (res, u) in zip(reqs, results):
        assert res["status"] == 0 and res["steps_done"] == q["nsteps"]
        assert _rel(u, _solo(mb4, q, precision="mixed")) <= 1e-12
        by_h.setdefault(q["h"], []).append((res["admitted"], res["completed"]))
    for spans in by_h.values():        # one slot fits: a class never runs two requests at once
        spans.sort()
        for a, b in zip(spans, spans[1:]):
            assert b[0] >= a[1] - 1e-9


def test_request_larger_than_budget_is_rejected(mb4):
    V = np.zeros(64 * 64)
    psi = inputs.wavepacket(64, 64, 4.0, 0.0, 0.0)
    with mb4.Server(1 << 16, max_slots=2) as srv:
        with pytest.raises(mb4.MB4Error) as e:
            srv.submit(64, 64, V, 1.0, psi, 0.01, 10)
        assert e.value.code == mb4.MB4_ERR_ADMISSION_REJECTED


def test_request_outside_its_class_fails_alone(mb4):
    """In an FP64 server the Krylov basis of a class is scaled by its x hopping, so a
    potential whose Gershgorin bound exceeds 4096 |tx| cannot join the class: that request
    ends with MB4_ERR_INVALID_ARG while the others run to completion.  Non-finite inputs
    are refused at submission."""
    reqs = _trace(3, seed=5, span=0.0)
    bad = dict(reqs[1])
    bad["V"] = bad["V"].copy()
    bad["V"][3] = 1.0e4
    reqs[1] = bad
    with mb4.Server(1 << 30, max_slots=4, keep_states=True, precision="fp64") as srv:
        ids = [srv.submit(q["nx"], q["ny"], q["V"], q["chi"], q["psi"], q["h"], q["nsteps"], q["arrival"])
               for q in reqs]
        nan_psi = reqs[0]["psi"].copy()
        nan_psi[0] = np.nan
        with pytest.raises(mb4.MB4Error) as e:
            srv.submit(reqs[0]["nx"], reqs[0]["ny"], reqs[0]["V"], 1.0, nan_psi, 0.01, 3)
        assert e.value.code == mb4.MB4_ERR_INVALID_ARG
        assert srv.run() == 3
        res = [srv.result(i) for i in ids]
    assert res[1]["done"] == 1 and res[1]["status"] == mb4.MB4_ERR_INVALID_ARG and res[1]["steps_done"] == 0
    for k in (0, 2):
        assert res[k]["status"] == mb4.MB4_OK and res[k]["steps_done"] == reqs[k]["nsteps"]
