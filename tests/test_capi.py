"""The C-ABI library builds, loads and exports every entry point of include/ipeps.h (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ipeps.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ipeps_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g

    g.build()
    return ctypes.CDLL(os.path.join(ROOT, "paper_2511_09546_gb300", "libipeps.so"))


def test_header_declares_the_hot_path():
    names = _declared()
    for must in ("ipeps_ctmrg", "ipeps_energy_grad", "ipeps_precondition", "ipeps_precondition_bp", "ipeps_optimize",
                 "ipeps_ham_create", "ipeps_env_destroy", "ipeps_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    # Hamiltonian assembly (S0) and option defaults run on the host
    from paper_2511_09546_gb300 import ipeps

    h = ipeps.ham_heisenberg(True)
    k = ipeps.ham_kitaev(-1.0)
    o = ipeps.default_opts(chi=32)
    assert o.chi == 32 and o.krylov == 30 and o.restarts == 1 and o.history == 200
    with pytest.raises(ipeps.IpepsError):
        ipeps.ham_create(2, [[float("nan")] * 4] * 4, [[0.0] * 4] * 4)
    del h, k


def test_nnn_setter_host_logic(lib):
    # the J1-J2 diagonal operators are attached on the host; bad input is reported
    import numpy as np

    from paper_2511_09546_gb300 import ipeps

    h = ipeps.ham_j1j2(1.0, 0.4, True)
    ipeps.ham_set_nnn(h, None, np.eye(4))      # one diagonal only
    ipeps.ham_set_nnn(h, None, None)           # removes both
    with pytest.raises(ipeps.IpepsError):
        ipeps.ham_set_nnn(h, np.full((4, 4), np.inf), None)
    st = ipeps.lib().ipeps_ham_set_nnn(None, None, None)
    assert st == 1 and b"NULL" in ipeps.lib().ipeps_last_error()
    del h


def test_job_footprint_host_logic(lib):
    # the server's admission estimate grows with (chi D^2)^2 and the cell size;
    # invalid shapes give 0
    from paper_2511_09546_gb300 import ipeps

    a = ipeps.job_footprint(1, 1, 2, 4, 32)
    b = ipeps.job_footprint(1, 1, 2, 4, 64)
    c = ipeps.job_footprint(2, 2, 2, 4, 64)
    assert 0 < a < b < c
    assert 3.0 < (b - (64 << 20)) / (a - (64 << 20)) < 4.5
    assert ipeps.job_footprint(0, 1, 2, 4, 64) == 0


def test_precondition_bp_argument_checks_on_host(lib):
    # the mean-field preconditioner rejects bad arguments before any device work
    import ctypes as C

    from paper_2511_09546_gb300 import ipeps

    L = ipeps.lib()
    sh = ipeps.Shape(1, 1, 2, 2)
    out = C.c_void_p(16)
    st = L.ipeps_precondition_bp(None, None, None, -1.0, 1e-12, 100, None, None, None, None)
    assert st == 1 and b"shape" in L.ipeps_last_error()
    st = L.ipeps_precondition_bp(C.byref(sh), None, None, -1.0, 1e-12, 100, out, None, None, None)
    assert st == 1 and b"NULL" in L.ipeps_last_error()
    big = ipeps.Shape(1, 1, 2, 33)
    st = L.ipeps_precondition_bp(C.byref(big), C.c_void_p(8), C.c_void_p(16), -1.0, 1e-12, 100,
                                 C.c_void_p(24), None, None, None)
    assert st == 1 and b"above 32" in L.ipeps_last_error()
    st = L.ipeps_precondition_bp(C.byref(sh), C.c_void_p(8), C.c_void_p(16), float("nan"), 1e-12, 100,
                                 C.c_void_p(24), None, None, None)
    assert st == 1 and b"finite" in L.ipeps_last_error()
    st = L.ipeps_precondition_bp(C.byref(sh), C.c_void_p(8), C.c_void_p(16), 0.1, 1e-12, 0,
                                 C.c_void_p(24), None, None, None)
    assert st == 1 and b"sweep" in L.ipeps_last_error()
    st = L.ipeps_precondition_bp(C.byref(sh), C.c_void_p(8), C.c_void_p(16), 0.1, 1e-12, 10,
                                 C.c_void_p(16), None, None, None)
    assert st == 1 and b"alias" in L.ipeps_last_error()


def test_optimize_rejects_unknown_preconditioner_on_host(lib):
    # precondition must be 0 (plain), 1 (local metric) or 2 (mean-field, D <= 32);
    # the options are checked before any device work
    import ctypes as C

    from paper_2511_09546_gb300 import ipeps

    L = ipeps.lib()
    h = ipeps.ham_heisenberg(True)
    for pre, D in ((3, 2), (-1, 2), (2, 33)):
        o = ipeps.default_opts(chi=8, precondition=pre)
        sh = ipeps.Shape(1, 1, 2, D)
        st = L.ipeps_optimize(C.byref(sh), C.c_void_p(8), h.h, C.byref(o), ipeps.ITER_CB(0), None, None)
        assert st == 1 and b"bad options" in L.ipeps_last_error(), (pre, D)


def test_public_header_is_plain_c():
    # the boundary is a C ABI: the header compiles as C99 (and as C++) on its own
    import os
    import shutil
    import subprocess

    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ipeps.h")
    for cc, args in (("gcc", ["-std=c99", "-x", "c"]), ("g++", ["-std=c++17", "-x", "c++"])):
        if shutil.which(cc) is None:
            pytest.skip(f"{cc} not installed")
        r = subprocess.run([cc, "-fsyntax-only", "-Wall", "-Werror", *args, hdr], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
