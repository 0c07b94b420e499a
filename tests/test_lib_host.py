"""Host-side checks of libmb4 that need no GPU: the library loads, exports every
entry point include/mb4.h declares, computes the MB4 constants correctly on the
host, and fails loudly (no CPU fallback) when no GPU is present."""
import os
import re
from fractions import Fraction

import numpy as np
import pytest

from oracle import mb4_oracle as orc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mb4():
    from paper_2003_04345_gb300 import build, mb4 as m
    if not os.path.exists(m.LIB_PATH):
        build.build()
    return m


def _declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mb4_[a-z0-9_]+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(mb4):
    L = mb4.lib()
    declared = _declared_entry_points()
    assert declared, "no entry points found in include/"
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing
    assert set(mb4.EXPORTS) <= declared


def test_library_constants_match_exact_ones(mb4):
    k = mb4.constants()
    E_exact, _ = orc.constants_f64()
    assert np.max(np.abs(k["E"] - E_exact)) < 4e-15 * np.max(np.abs(E_exact))
    lam_oracle = np.sort(np.linalg.eigvals(E_exact[:, 1:]).real)
    assert np.max(np.abs(k["lam"] - lam_oracle)) < 1e-14
    assert np.all(np.diff(k["lam"]) > 0)
    T, Ti = k["T"], k["Tinv"]
    assert np.max(np.abs(T @ Ti - np.eye(3))) < 1e-14
    assert np.max(np.abs(T @ np.diag(k["lam"]) @ Ti - E_exact[:, 1:])) < 1e-13
    assert np.allclose(np.linalg.norm(T, axis=0), 1.0, atol=1e-15)


def test_library_gauss_rule_is_exact_to_degree_11(mb4):
    k = mb4.constants()
    x, w = k["gauss_x"], k["gauss_w"]
    for deg in range(12):
        assert abs(np.sum(w * x ** deg) - 1.0 / (deg + 1)) < 2e-16 * 8
    assert abs(np.sum(w * x ** 12) - 1.0 / 13) > 1e-8   # and not beyond (6 nodes)


def test_library_constants_other_nodes(mb4):
    k = mb4.constants(-712.5, 0.25, 0.5)
    E_exact, _ = orc.constants_f64(Fraction(-5700, 8), (Fraction(1, 4), Fraction(1, 2), Fraction(1)))
    assert np.max(np.abs(k["E"] - E_exact)) < 4e-15 * np.max(np.abs(E_exact))


def test_library_rejects_alpha_above_bound(mb4):
    with pytest.raises(mb4.MB4Error) as e:
        mb4.constants(-200.0)
    assert e.value.code == mb4.MB4_ERR_INVALID_ARG


def test_create_fails_loudly_without_gpu(mb4):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(mb4.MB4Error) as e:
        mb4.Integrator(4, 4, np.zeros(16), 1.0, 0.01)
    assert e.value.code == mb4.MB4_ERR_CUDA


def test_status_strings(mb4):
    assert mb4.status_string(0) == "ok"
    assert "Newton" in mb4.status_string(mb4.MB4_ERR_NEWTON_NOT_CONVERGED)


def _build_c_demo(tmp_path):
    """Compile tests/c/abi_demo.c with the host C compiler against include/mb4.h and
    the in-tree libmb4.so (found at run time through its rpath)."""
    import shutil
    import subprocess
    from paper_2003_04345_gb300 import mb4 as m
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib_dir = os.path.dirname(m.LIB_PATH)
    exe = str(tmp_path / "abi_demo")
    subprocess.run([cc, "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_demo.c"), "-o", exe, "-L", lib_dir, "-lmb4",
                    f"-Wl,-rpath,{lib_dir}", "-lm"], check=True)
    return exe


def test_c_program_uses_the_abi_and_fails_loudly_without_gpu(mb4, tmp_path):
    """A plain C program compiles against include/mb4.h, links libmb4.so and, with no
    GPU, gets MB4_ERR_CUDA from mb4_create (exit status 3): no CPU fallback."""
    import subprocess
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present: the GPU test runs the program")
    except ImportError:
        pass
    exe = _build_c_demo(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 3, (r.returncode, r.stdout, r.stderr)
    assert "mb4_create" in r.stdout


@pytest.mark.gpu
def test_c_program_steps_and_conserves_energy(mb4, tmp_path):
    """The same C program on a GPU: 100 steps, |dH/H| <= 1e-13 (exit status 0)."""
    import subprocess
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    exe = _build_c_demo(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert "steps 100" in r.stdout


def test_batch_bytes_counts_the_planes_a_batch_allocates(mb4):
    """mb4_batch_bytes (host arithmetic, no GPU): at least the per-site planes a batch
    allocates -- u 16, V 8, onsite+V 8, D/tx 8, (K+V)u0 16, dU 48, J 4 tk, basis
    (s+1) 6 tk, two history steps 96 -- linear in the batch, and smaller in mixed mode."""
    S = 512 * 512
    for precision, tk in (("fp64", 8), ("mixed", 4)):
        per_site = 16 + 8 + 8 + 8 + 16 + 48 + 4 * tk + 5 * 6 * tk + 96
        one = mb4.batch_bytes(512, 512, 1, precision=precision)
        assert one >= per_site * S
        assert mb4.batch_bytes(512, 512, 4, precision=precision) >= 4 * per_site * S
    assert mb4.batch_bytes(512, 512, 1, precision="mixed") < mb4.batch_bytes(512, 512, 1, precision="fp64")
    assert mb4.batch_bytes(2, 512, 1) == -1


def test_binding_structs_match_the_header(mb4, tmp_path):
    """Every ctypes struct of the binding has the size and field offsets of its C typedef in
    include/mb4.h (compiled here by the host C compiler): a field added to, moved in or
    renamed in the header without the binding fails here, on the CPU."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [(mb4.Grid, "mb4_grid"), (mb4.Potential, "mb4_potential"), (mb4.Nonlinearity, "mb4_nonlinearity"),
             (mb4.SparseKinetic, "mb4_sparse_kinetic"), (mb4.Options, "mb4_options"), (mb4.Stats, "mb4_stats"),
             (mb4.Request, "mb4_request"), (mb4.Result, "mb4_result")]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "mb4.h"', "int main(void) {"]
    want = []
    for cls, cname in pairs:
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        want.append(ctypes.sizeof(cls))
        for name, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {name}));')
            want.append(getattr(cls, name).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", exe],
                   check=True)
    got = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert got == want
