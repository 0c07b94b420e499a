"""mb4_observables_noalloc: the observables of a state for callers that cannot
allocate device memory (code under an allocator that owns all device memory,
or where cudaMalloc and its implicit synchronisation are not allowed).

The entry point keeps its block partial sums in a fixed array inside the
library instead of allocating.  Through the C ABI it must give the same six
observables as the context-based mb4_observables, call after call, although
every call reuses the same scratch array, and match the FP64 oracle's correctly rounded
sums.  This file is collected last so that
a run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2003_04345_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 2e-15   # the relative tolerance of the observables tests


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2003_04345_gb300 import mb4
    mb4.lib()
    return torch, mb4


def _context_observables(mb4, nx, ny, V, chi, tx, ty, onsite, psi):
    with mb4.Integrator(nx, ny, V, chi, 0.01, tx=tx, ty=ty, onsite=onsite) as it:
        it.set_state(psi)
        o = it.observables()
    return np.array([o["H"], o["U_K"], o["U_E"], o["U_nl"], o["norm2"], o["participation"]])


def _close(got, want):
    return np.all(np.abs(got - want) <= TOL * np.maximum(np.abs(want), 1e-300) + 1e-18)


@pytest.mark.parametrize("nx,ny", [(16, 16), (129, 77)])
def test_noalloc_matches_context_observables_twice(env, nx, ny):
    torch, mb4 = env
    S = nx * ny
    rng = np.random.default_rng(nx * ny)
    V = inputs.potential(nx, ny, 1.0, max(1, S // 100), 20.0, 5)
    chi, tx, ty, onsite = 1.3, 1.0, 0.8, 0.2
    states = [inputs.wavepacket(nx, ny, 3.0, np.pi / 4, 0.0),
              0.1 * (rng.normal(size=S) + 1j * rng.normal(size=S))]
    Vd = torch.tensor(V, dtype=torch.float64, device="cuda")
    out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for psi in states:            # two calls in a row on different states share the scratch
        want = _context_observables(mb4, nx, ny, V, chi, tx, ty, onsite, psi)
        re = torch.tensor(psi.real.copy(), dtype=torch.float64, device="cuda")
        im = torch.tensor(psi.imag.copy(), dtype=torch.float64, device="cuda")
        rc = mb4.lib().mb4_observables_noalloc(nx, ny, tx, ty, onsite, chi, re.data_ptr(), im.data_ptr(),
                                               Vd.data_ptr(), out.data_ptr(), stream.cuda_stream)
        assert rc == mb4.MB4_OK, mb4.status_string(rc)
        stream.synchronize()
        got = out.cpu().numpy()
        assert _close(got, want), (got, want)
        # and against the FP64 oracle's correctly rounded sums directly
        from oracle import mb4_oracle as orc
        prob = orc.Problem(nx, ny, V, chi, tx=tx, ty=ty, eps0=onsite)
        H, UK, UE, UI = orc.energy(prob, psi)
        ref = np.array([H, UK, UE, UI, orc.norm2(psi), orc.participation(psi)])
        scale = np.array([abs(UK) + abs(UE) + abs(UI)] * 4 + [ref[4], ref[5]])
        assert np.all(np.abs(got - ref) <= 1e-14 * scale), (got, ref)


def test_noalloc_allocates_nothing(env):
    """Repeated calls leave the device's free memory and torch's allocator untouched: the
    entry point uses only its fixed array, never cudaMalloc.  Measured after a first call,
    so that the one-time loading of the library's kernels onto the device is not counted."""
    torch, mb4 = env
    nx, ny = 96, 80
    S = nx * ny
    psi = inputs.wavepacket(nx, ny, 4.0, np.pi / 4, 0.0)
    V = torch.tensor(inputs.potential(nx, ny, 1.0, S // 100, 20.0, 9), dtype=torch.float64, device="cuda")
    re = torch.tensor(psi.real.copy(), dtype=torch.float64, device="cuda")
    im = torch.tensor(psi.imag.copy(), dtype=torch.float64, device="cuda")
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    L = mb4.lib()

    def call():
        rc = L.mb4_observables_noalloc(nx, ny, 1.0, 1.0, 0.0, 1.0, re.data_ptr(), im.data_ptr(), V.data_ptr(),
                                       out.data_ptr(), stream.cuda_stream)
        assert rc == mb4.MB4_OK, mb4.status_string(rc)

    call()
    stream.synchronize()
    first = out.cpu().numpy().copy()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(5):
        call()
    stream.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0, (free0, free1)
    assert np.array_equal(out.cpu().numpy(), first)      # same inputs, same fixed-order sums


def test_noalloc_rejects_out_of_range_sizes(env):
    torch, mb4 = env
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    L = mb4.lib()
    assert L.mb4_observables_noalloc(2, 8, 1.0, 1.0, 0.0, 1.0, x.data_ptr(), x.data_ptr(), x.data_ptr(),
                                     x.data_ptr(), None) == mb4.MB4_ERR_INVALID_ARG
    # 65536 x 32768 sites exceeds MB4_NOALLOC_MAX_SITES; rejected before any launch
    assert L.mb4_observables_noalloc(65536, 32768, 1.0, 1.0, 0.0, 1.0, x.data_ptr(), x.data_ptr(),
                                     x.data_ptr(), x.data_ptr(), None) == mb4.MB4_ERR_INVALID_ARG
