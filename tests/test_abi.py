"""Host-side checks of the C ABI that need no GPU: the library builds for sm_103a, loads,
and exports every function include/cvba.h declares; status strings; a context cannot be
created without a GB300 (no silent CPU path)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_04359_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^\s*(?:const\s+)?[\w]+\*?\s+\*?(cvba_\w+)\s*\(", src, re.M)
    return sorted(set(names))


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ["cvba_create", "cvba_set_rig", "cvba_set_poses", "cvba_set_landmarks", "cvba_set_observations",
              "cvba_solve", "cvba_get_poses", "cvba_get_landmarks", "cvba_get_increment", "cvba_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    lib.cvba_status_string.restype = ctypes.c_char_p
    assert lib.cvba_status_string(0) == b"ok"
    assert lib.cvba_status_string(2) == b"index out of range"
    assert lib.cvba_status_string(99) == b"unknown status"


def test_binding_loads_and_matches_struct_layout(lib, tmp_path):
    """The ctypes structs and the trace dtype match the C header's layout (sizes and every
    field offset, as compiled by the host C compiler)."""
    import shutil
    import subprocess
    from paper_2506_04359_gb300 import cvba
    assert cvba.ITER_DTYPE.itemsize == ctypes.sizeof(cvba.cvba_iter)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"cvba_opts": cvba.cvba_opts, "cvba_iter": cvba.cvba_iter}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cvba.h"', "int main(void) {"]
    for name, py in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in py._fields_:
            cf = "lambda" if f == "lambda_" else f
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {cf}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for line in filter(None, out):
        name, field, val = line.split()
        py = structs[name]
        got = ctypes.sizeof(py) if field == "size" else getattr(py, field).offset
        assert got == int(val), (name, field)
    for f in cvba.ITER_DTYPE.names:
        cf = "lambda_" if f == "lambda" else f
        assert cvba.ITER_DTYPE.fields[f][1] == getattr(cvba.cvba_iter, cf).offset


def test_create_fails_loudly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2506_04359_gb300 import cvba
    with pytest.raises(cvba.CvbaError):
        cvba.Context("fp64")


def test_oracle_device_layout_definition():
    """The layout definition the GPU is checked against, on a brute-force example."""
    from oracle import ba
    rng = np.random.default_rng(3)
    N, M, K = 300, 25, 7
    kf, cam, lm = rng.integers(0, K, N), rng.integers(0, 4, N), rng.integers(0, M, N)
    lo, oo, off = ba.device_layout(kf, cam, lm, M)
    first = [min(kf[lm == j], default=10 ** 9) for j in range(M)]
    last = [max(kf[lm == j], default=-1) for j in range(M)]
    ref_lo = sorted(range(M), key=lambda j: (first[j], last[j], j))
    assert lo.tolist() == ref_lo
    rank = {j: r for r, j in enumerate(ref_lo)}
    ref_oo = sorted(range(N), key=lambda n: (rank[lm[n]], kf[n], cam[n], n))
    assert oo.tolist() == ref_oo
    assert off[-1] == N and all(off[r + 1] - off[r] == int((lm == ref_lo[r]).sum()) for r in range(M))


def _declared_arity():
    """Parameter count of every function declared in include/*.h."""
    out = {}
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", f)).read(), flags=re.S)
        for m in re.finditer(r"(cvba_\w+)\s*\(([^;{]*?)\)\s*;", src):
            args = m.group(2).strip()
            out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_signatures_match_the_header(lib):
    """Every function the ctypes binding declares takes as many arguments as the header says."""
    from paper_2506_04359_gb300 import cvba
    arity = _declared_arity()
    for name, n in arity.items():
        f = getattr(cvba.lib, name, None)
        if f is None or f.argtypes is None:
            continue
        assert len(f.argtypes) == n, (name, len(f.argtypes), n)
