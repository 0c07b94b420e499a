"""The persistent step kernel (option persistent = 1): one cooperative launch per step
holding the set-up and the whole Newton loop, its phases separated by bounded grid
barriers.  It runs the same device code over the same data as the graph step, so the
two give the same states and the same Newton counts bit for bit; its waits end with
MB4_ERR_TIMEOUT instead of hanging, and the state then stays at the last accepted step."""
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


def _run(mb4, w, steps, chunk=1, **opts):
    with mb4.from_workload(w, **opts) as it:
        total = 0
        for _ in range(steps // chunk):
            total += it.step(chunk)["newton_iters_total"]
        return it.get_state(), total, it.observables()


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("s", [4, 5])
def test_persistent_equals_graph_bit_for_bit_grid16(mb4, precision, s):
    """16 x 16 workload, 100 steps in chunks of 7 (steps that start from both Newton
    starts): state, Newton iterations and observables identical to the graph step, and
    the state on the oracle's to 1e-11."""
    w = inputs.grid16_fp64()
    a, na, oa = _run(mb4, w, 98, chunk=7, precision=precision, krylov_s=s)
    b, nb, ob = _run(mb4, w, 98, chunk=7, precision=precision, krylov_s=s, persistent=1)
    assert np.array_equal(a, b)
    assert na == nb
    assert oa == ob
    prob = orc.Problem(w.nx, w.ny, w.potential(), w.chi, tx=w.tx, ty=w.ty, eps0=w.eps0)
    u, _ = orc.run(prob, w.psi0(), w.h, 98)
    assert np.max(np.abs(b - u)) <= 1e-11 * np.max(np.abs(u))


@pytest.mark.parametrize("precision", PRECISIONS)
def test_persistent_equals_graph_bit_for_bit_grid512(mb4, precision):
    """The 512 x 512 benchmark workload, 12 steps: identical to the graph step."""
    w = inputs.grid512_fp64()
    a, na, _ = _run(mb4, w, 12, chunk=4, precision=precision)
    b, nb, _ = _run(mb4, w, 12, chunk=4, precision=precision, persistent=1)
    assert np.array_equal(a, b)
    assert na == nb


@pytest.mark.parametrize("precision", PRECISIONS)
def test_persistent_equals_graph_other_stencils_and_chi_field(mb4, precision):
    """tx = 0 (the stencil without the factored x hopping), and a per-site chi field: the
    other kernel variants of the persistent step, identical to the graph step."""
    rng = np.random.default_rng(3)
    nx, ny = 40, 24
    S = nx * ny
    V = inputs.potential(nx, ny, 1.0, 5, 20.0, 4)
    psi = inputs.wavepacket(nx, ny, 3.0, np.pi / 4, 0.3)
    chi = rng.uniform(0.0, 2.0, S)
    for tx, field in ((0.0, False), (0.9, True)):
        states = []
        for persistent in (0, 1):
            with mb4.Integrator(nx, ny, V, 1.0, 0.01, tx=tx, ty=1.1, onsite=0.2, precision=precision,
                                site_chi=field, persistent=persistent) as it:
                if field:
                    it.set_chi_field(chi)
                it.set_state(psi)
                it.step(20)
                states.append(it.get_state())
        assert np.array_equal(states[0], states[1]), (tx, field)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_persistent_batch_equals_graph_batch(mb4, precision):
    """A batch of 6 instances with different potentials and chi: identical to the graph
    batch, instance by instance (an instance converges and is masked while others go on)."""
    n, B = 32, 6
    ws = [inputs.ensemble128(seed) for seed in range(B)]
    V = np.stack([inputs.potential(n, n, 1.0, 10, 20.0, seed) for seed in range(B)])
    chi = np.array([w.chi for w in ws])
    psi = np.stack([inputs.wavepacket(n, n, 3.0 + b, np.pi / 4, 0.0) for b in range(B)])
    out = []
    for persistent in (0, 1):
        with mb4.Batch(n, n, V, chi, 0.01, precision=precision, persistent=persistent) as bt:
            bt.set_state(psi)
            stats, codes = bt.step(30)
            assert not any(codes)
            out.append((bt.get_state(), [s["newton_iters_total"] for s in stats]))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


@pytest.mark.parametrize("precision", PRECISIONS)
def test_persistent_wait_limit_zero_times_out_and_keeps_the_state(mb4, precision):
    """wait_limit = 0: a grid-barrier wait gives up at its first poll.  The step returns
    MB4_ERR_TIMEOUT (no hang, no fault), the state stays at the last accepted step, and
    the context stays usable: observables, and a following call that times out again.
    (64 x 64, so that the step runs on several blocks: one block alone never waits.)"""
    w = inputs.Workload("grid64", 64, 64, h=0.01, steps=10, chi=1.0, W=1.0, defect_fraction=0.01, sigma=4.0)
    with mb4.from_workload(w, precision=precision, persistent=1, wait_limit=0) as it:
        u0 = it.get_state()
        H0 = it.energy()[0]
        st, rc = it.step(3, check=False)
        assert rc == mb4.MB4_ERR_TIMEOUT, mb4.status_string(rc)
        assert st["steps_done"] == 0
        assert np.array_equal(it.get_state(), u0)
        assert it.energy()[0] == H0
        st, rc = it.step(1, check=False)
        assert rc == mb4.MB4_ERR_TIMEOUT
        assert np.array_equal(it.get_state(), u0)
    # and a context with the default limit on the same device steps normally afterwards
    a, _, _ = _run(mb4, w, 5, precision=precision, persistent=1)
    b, _, _ = _run(mb4, w, 5, precision=precision)
    assert np.array_equal(a, b)


def test_persistent_refused_where_it_has_no_kernel(mb4):
    n = 32
    V = np.zeros(n * n)
    tx, ty, e0 = inputs.paper_laplacian_hopping(n, n)
    with pytest.raises(mb4.MB4Error) as e:
        mb4.Integrator(n, n, V, -0.1, 0.01, tx=tx, ty=ty, onsite=e0, precondition=1, persistent=1)
    assert e.value.code == mb4.MB4_ERR_INVALID_ARG
    with pytest.raises(mb4.MB4Error) as e:
        mb4.Integrator(n, n, V, 1.0, 0.01, krylov_s=3, persistent=1)
    assert e.value.code == mb4.MB4_ERR_INVALID_ARG
    K = np.diag(np.ones(9), 1) + np.diag(np.ones(9), -1)
    with pytest.raises(mb4.MB4Error) as e:
        mb4.Integrator.sparse(K, np.zeros(10), 1.0, 0.01, persistent=1)
    assert e.value.code == mb4.MB4_ERR_INVALID_ARG
