"""Long oracle trajectories for the GPU parity tests, computed in spawned processes.

The oracle needs minutes for the longest comparisons (the 128 x 128 case with the
2048 x 2048 physics over its 500 steps, the paper's 70 x 70 run over 30 steps and its
delta-potential run over 20).  conftest.py starts these jobs in a spawn-context process
pool as soon as a session selects a test marked ``oracle_long``, so they run on the host
cores while the other GPU tests use the GPU; a test then waits for its job's result.
Each job imports only the oracle and the input generators (never torch or the CUDA
binding), and returns plain numpy arrays.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp

import numpy as np

PAPER_RTOL = 2e-14      # the paper's absolute 1e-13 (Sec. 3) at the initial peak |u0| = 5


def c3_crop(checkpoints=(10, 100, 250, 500)):
    """128 x 128 instance with the 2048 x 2048 physics (W = 2, chi = 2, 1% defects,
    h = 0.002): states at the checkpoints and H every 10 steps."""
    from oracle import mb4_oracle as orc
    from paper_2003_04345_gb300 import inputs
    w = inputs.grid128_crop_of_2048()
    prob = orc.Problem(w.nx, w.ny, w.potential(), w.chi, tx=w.tx, ty=w.ty, eps0=w.eps0)
    u = w.psi0()
    out = {"H": [orc.energy(prob, u)[0]]}
    for n in range(1, max(checkpoints) + 1):
        u = orc.step(prob, u, w.h)
        if n in checkpoints:
            out[n] = u.copy()
        if n % 10 == 0:
            out["H"].append(orc.energy(prob, u)[0])
    return out


def _paper_problem(n, gamma, V0):
    from oracle import mb4_oracle as orc
    from paper_2003_04345_gb300 import inputs
    tx, ty, e0 = inputs.paper_laplacian_hopping(n, n)
    V = np.zeros(n * n) if V0 is None else inputs.delta_potential(n, n, V0)
    prob = orc.Problem(n, n, V, -gamma, tx=tx, ty=ty, eps0=e0)
    return orc, prob, inputs.paper_initial_state(n, n)


def paper70(nsteps=30, checkpoints=(3, 10, 30)):
    """The paper's 70 x 70 run (gamma = 0.1, h = 0.01, Sec. 3): states at the checkpoints."""
    orc, prob, u = _paper_problem(70, 0.1, None)
    out = {}
    for n in range(1, nsteps + 1):
        u = orc.step(prob, u, 0.01, solver="lu")
        if n in checkpoints:
            out[n] = u.copy()
    return out


def delta100(nsteps=20):
    """The paper's delta-potential run (Sec. 3.2: 100 x 100, gamma = 0.05, V0 = -50,
    h = 0.01): after every step the observables (H, U_K, U_E, U_I, participation ratio),
    and the states after 2, 10 and 20 steps."""
    orc, prob, u = _paper_problem(100, 0.05, -50.0)
    out = {"obs": []}

    def obs(v):
        H, UK, UE, UI = orc.energy(prob, v)
        return [H, UK, UE, UI, orc.participation(v)]
    out["obs"].append(obs(u))
    for n in range(1, nsteps + 1):
        u = orc.step(prob, u, 0.01, solver="lu")
        out["obs"].append(obs(u))
        if n in (2, 10, nsteps):
            out[n] = u.copy()
    out["obs"] = np.array(out["obs"])
    return out


JOBS = {"c3_crop": c3_crop, "paper70": paper70, "delta100": delta100}

_pool = None
_futures = {}


def start(names=tuple(JOBS)):
    """Submit the named jobs to a spawn-context pool (idempotent)."""
    global _pool
    if _pool is None:
        _pool = cf.ProcessPoolExecutor(max_workers=len(JOBS), mp_context=mp.get_context("spawn"))
    for name in names:
        if name not in _futures:
            _futures[name] = _pool.submit(JOBS[name])


def result(name):
    """The job's result, starting it (in this session's pool) if nobody has yet."""
    if name not in _futures:
        start((name,))
    return _futures[name].result()


def shutdown():
    """Stop the pool; jobs still running (a session that stopped early) are terminated."""
    global _pool
    if _pool is not None:
        procs = list(getattr(_pool, "_processes", {}).values())
        _pool.shutdown(wait=False, cancel_futures=True)
        for p in procs:
            if p.is_alive():
                p.terminate()
        _pool = None
        _futures.clear()
