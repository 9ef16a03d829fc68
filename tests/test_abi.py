"""The C ABI loads and exports every symbol include/coilsketch.h declares; host-side library
code (Philox known answers, the FP64 Jacobi eigensolver that coil_pca runs on the GPU) is
checked without a GPU.  No compute call touches a device here."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cs():
    import __graft_entry__ as g
    from paper_2305_06482_gb300 import build as b
    b.build()
    import paper_2305_06482_gb300 as cs
    cs.lib()
    return cs


def _declared():
    src = open(os.path.join(ROOT, "include", "coilsketch.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:[a-z_0-9]+\s+)+\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(cs):
    names = _declared()
    assert "recon_solve" in names and "sense_fwd" in names and "coil_pca" in names
    assert "cs_launch_count" in names and "cs_hermitian_eig_host" in names
    L = cs.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(cs.EXPORTED)


def test_version_and_error_string(cs):
    assert b"sm_103a" in cs.lib().cs_version()


def _kat():
    rows = []
    for line in open(os.path.join(ROOT, "tests", "golden", "philox4x32_10_kat.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            w = [int(t, 16) for t in line.split()]
            rows.append((tuple(w[0:4]), tuple(w[4:6]), tuple(w[6:10])))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat())
def test_library_philox_known_answers(cs, ctr, key, want):
    assert cs.philox4x32_10(ctr, key) == want


def test_library_philox_matches_oracle_generator(cs):
    from oracle import philox
    rng = np.random.default_rng(0)
    for _ in range(50):
        ctr = tuple(int(v) for v in rng.integers(0, 2 ** 32, 4))
        key = tuple(int(v) for v in rng.integers(0, 2 ** 32, 2))
        assert cs.philox4x32_10(ctr, key) == philox.philox4x32_10(ctr, key)


@pytest.mark.parametrize("n", [1, 2, 5, 8, 20, 40])
def test_jacobi_eigensolver_host(cs, n):
    rng = np.random.default_rng(n)
    Y = rng.standard_normal((n, 3 * n + 5)) + 1j * rng.standard_normal((n, 3 * n + 5))
    Y *= np.linspace(3, 0.1, n)[:, None]
    A = Y @ Y.conj().T
    V, ev = cs.hermitian_eig_host(A)
    w = np.linalg.eigvalsh(A)[::-1]
    assert np.allclose(ev, w, rtol=1e-12, atol=1e-12 * w[0])
    assert np.allclose(V.conj().T @ V, np.eye(n), atol=1e-12)
    assert np.allclose(A @ V, V * ev[None, :], atol=1e-10 * w[0])
    j = np.argmax(np.abs(V), axis=0)
    piv = V[j, np.arange(n)]
    assert np.all(piv.imag == 0) and np.all(piv.real > 0)


def test_jacobi_degenerate_spectrum(cs):
    rng = np.random.default_rng(9)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6)))
    ev = np.array([5, 5, 2, 2, 2, 0.5])
    A = (Q * ev) @ Q.conj().T
    V, got = cs.hermitian_eig_host(A)
    assert np.allclose(got, ev, atol=1e-12)
    # projector onto the top-2 eigenspace is unique even though the vectors are not
    P1 = V[:, :2] @ V[:, :2].conj().T
    P2 = Q[:, :2] @ Q[:, :2].conj().T
    assert np.allclose(P1, P2, atol=1e-12)


def test_host_side_argument_checks(cs):
    """Entry points refuse bad arguments on the host, before any device work (no GPU needed)."""
    import ctypes
    L = cs.lib()
    i3 = ctypes.c_int * 3
    fake = ctypes.c_void_p(0x1000)       # never dereferenced: the checks fail first
    assert L.cs_plan_set_gridding(None, 16, 64, 16, 64) == 1
    assert L.cs_plan_autotune(None, 4, 3, None, None, None) == 1
    assert L.cs_wait_selftest(0, 0, None) == 1                       # poll limit out of range
    assert L.cs_wait_selftest(0, (1 << 24) + 1, None) == 1
    h = ctypes.c_void_p()
    assert L.ws_net_create(6, 16, 32, ctypes.c_uint64(0), ctypes.byref(h)) == 2   # width not a multiple of 4
    assert L.ws_net_create(16, 64, 64, ctypes.c_uint64(0), ctypes.byref(h)) == 2  # concatenation too wide
    assert L.ws_net_create(16, 32, 64, ctypes.c_uint64(0), None) == 1
    assert L.ws_net_infer(None, fake, fake, i3(8, 8, 8), ctypes.c_float(1.0), fake, None) == 1
    assert L.cs_crop3d(fake, i3(8, 8, 8), i3(4, 0, 0), i3(8, 8, 8), fake, None) == 1  # box leaves the volume
    assert L.cs_crop3d(fake, i3(8, 8, 8), i3(-1, 0, 0), i3(4, 4, 4), fake, None) == 1
    assert b"crop box" in L.cs_last_error()


def test_ctypes_structs_match_the_c_layout(tmp_path):
    """Every struct of include/coilsketch.h that the binding mirrors has the same size and field
    offsets in C (compiled here with the host compiler) and in ctypes."""
    import ctypes
    import shutil
    import subprocess

    import paper_2305_06482_gb300 as cs

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    mirrors = {"cs_geom": cs._Geom, "cs_problem": cs._Problem, "cs_solve_params": cs._Params,
               "cs_stats": cs._Stats, "cs_batch_item": cs._BatchItem}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "coilsketch.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            cfield = "lambda" if fname == "lam" else fname
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {cfield}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(ROOT, "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln.strip():
            a, b, v = ln.split()
            got[(a, b)] = int(v)
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
