"""The C-ABI library loads and exports every symbol include/hemegb.h declares (CPU only);
the header is plain C99.

Also checks the one host-only entry point, hg_coupling_factors (Section 3's
coupling map and scale factors), against the oracle's implementation.
"""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hemegb.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(hg_\w+)\s*\(", src, re.M)))


def test_header_symbols_exported(hemegb_lib):
    names = _declared()
    assert len(names) >= 20
    L = hemegb_lib.lib()
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", hemegb_lib.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (hg_\w+)", out))
    assert set(names) <= exported
    # the binding wraps every declared function under the same name
    assert set(names) == set(hemegb_lib.exported_symbols())


def test_no_gpu_context_fails_cleanly(hemegb_lib):
    import torch

    if torch.cuda.is_available():
        return
    import ctypes as C

    p = hemegb_lib.hg_ctx_params()
    p.device, p.storage, p.scheme = 0, 0, 0
    h = C.c_void_p()
    rc = hemegb_lib.lib().hg_ctx_create(C.byref(p), C.byref(h))
    assert rc == hemegb_lib.HG_ERR_CUDA
    p.storage = 7
    assert hemegb_lib.lib().hg_ctx_create(C.byref(p), C.byref(h)) == hemegb_lib.HG_ERR_ARG


def test_coupling_factors_match_oracle(hemegb_lib):
    from oracle import coupling as CP

    g = np.random.default_rng(3)
    for trial in range(20):
        na = int(g.integers(1, 6))
        nv = int(g.integers(na, 13 * na + 1))
        art = [tuple(int(v) for v in g.integers(0, 200 * 1024, 3)) for _ in range(na)]
        ven = [tuple(int(v) for v in g.integers(0, 200 * 1024, 3)) for _ in range(nv)]
        if trial == 0:
            ven[1] = ven[0]  # a tie
        aa = list(1 + 50 * g.random(na))
        va = list(1 + 50 * g.random(nv))
        un = g.random(nv)
        assign, dist, dp, fac = hemegb_lib.hg_coupling_factors(art, aa, ven, va, un)
        ra, rd = CP.greedy_map(art, ven)
        assert list(assign) == ra
        np.testing.assert_allclose(dist, rd, rtol=1e-15)
        np.testing.assert_allclose(dp, CP.pressure_drops(un), rtol=1e-15)
        table = CP.coupling_table(art, aa, ven, va, un)
        ref = np.zeros(nv)
        for (a, v, L, d, f) in table:
            ref[v] = f
        np.testing.assert_allclose(fac, ref, rtol=1e-13)


def test_paper_example_through_abi(hemegb_lib):
    """1:3 example of Section 3 through the host helper (golden fixture)."""
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "coupling_1to3.txt"))
            if l.strip() and not l.startswith("#")]
    dP = np.array([float(r[1]) for r in rows])
    L = np.array([float(r[3]) for r in rows])
    # place three veins on a line at the given distances from one artery
    art = [(0, 0, 0)]
    ven = [(int(round(l * 1024)), 0, 0) for l in L]
    un = (dP - 0.3) / 0.4
    assign, dist, dp, fac = hemegb_lib.hg_coupling_factors(art, [1.0], ven, [1.0] * 3, un)
    assert list(assign) == [0, 0, 0]
    assert [round(f, 2) for f in fac] == [float(r[2]) for r in rows]


def test_header_is_plain_c(tmp_path):
    """include/hemegb.h compiles as strict C99 (a C ABI with no C++ or CUDA types)."""
    import shutil

    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    hdr = os.path.join(ROOT, "include", "hemegb.h")
    src = tmp_path / "use.c"
    src.write_text(f'#include "{hdr}"\nint main(void) {{ hg_ctx_params p = {{0}}; (void)p; return 0; }}\n')
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-c", str(src),
                        "-o", str(tmp_path / "use.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_every_declaration_cites_its_passage():
    """Each entry point's comment names the paper passage that defines the operation,
    or says that it is infrastructure with no passage (or has no counterpart)."""
    src = open(os.path.join(ROOT, "include", "hemegb.h")).read()
    decls = list(re.finditer(r"^\s*(?:int|const char \*)\s*(hg_\w+)\s*\(", src, re.M))
    assert len(decls) >= 20
    for m in decls:
        head = src[:m.start()].rstrip()
        assert head.endswith("*/"), m.group(1)
        comment = head[head.rfind("/*"):]
        line = [l for l in comment.splitlines() if "Passage:" in l]
        assert line, f"{m.group(1)} has no 'Passage:' line"
        text = comment[comment.find("Passage:"):]
        assert ("Section" in text or "Eq." in text or "infrastructure: no passage" in text
                or "no counterpart in the paper" in text), m.group(1)
