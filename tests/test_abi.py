"""Host-side checks of the C-ABI library: it builds for sm_103a, loads, exports
every entry point declared in include/*.h, and its host-only logic (size
queries, argument validation) behaves.  No GPU is touched."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b([a-z_][a-z0-9_]*)\s*\(", src):
            name = m.group(1)
            before = src[:m.start()].rstrip()
            if name in ("if", "while", "for", "sizeof", "return"):
                continue
            if before.endswith(("typedef", "(")):
                continue
            names.add(name)
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2312_09376_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("rbt_generate", "rbt_apply_2sided", "rbt_apply_vec", "genp_factor", "genp_solve",
                     "rbt_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_2312_09376_gb300 import _lib
    assert set(_declared_functions()) <= set(_lib.declared_symbols()) | {"rbt_status_string"}


def test_status_strings(lib):
    assert lib.rbt_status_string(0) == b"ok"
    assert lib.rbt_status_string(1) == b"zero pivot"
    assert lib.rbt_status_string(-1) == b"invalid argument"


def test_argument_validation_without_gpu(lib):
    P = ctypes.c_void_p
    assert lib.rbt_generate(-1, 2, 1, None, None, 1, None) == -1
    assert lib.rbt_generate(10, 2, 1, None, None, 5, None) == -1       # ldw < n
    assert lib.rbt_generate(10, 2, 1, None, None, 10, None) == -1      # null pointers
    assert lib.rbt_generate(0, 2, 1, None, None, 1, None) == 0         # empty: nothing to do
    assert lib.rbt_apply_2sided(10, 2, None, None, 10, None, 10, None, 10, None) == -1
    assert lib.rbt_apply_2sided(10, -1, P(8), P(8), 10, P(8), 10, P(8), 10, None) == -1
    assert lib.rbt_apply_2sided(10, 2, P(8), P(8), 10, P(8), 9, P(8), 10, None) == -1   # lda < n
    # partial overlap of input and output is refused before any launch
    assert lib.rbt_apply_2sided(10, 2, P(8), P(8), 10, P(4096), 10, P(4096 + 8), 10, None) == -1
    assert lib.rbt_apply_vec(10, 2, P(8), 10, 1, P(8), 3, 1, None) == -1
    assert lib.genp_solve(10, 1, 7, P(8), 10, 0, P(8), 10, None, 0, None) == -1         # bad precision


def test_workspace_queries(lib):
    from paper_2312_09376_gb300 import _lib
    for prec in ("f64", "f32"):
        o = _lib.make_opts(depth=2, prec=prec, fallback=True)
        ws = _lib.rbt_solve_workspace(o, 1003, 1)
        es = 8 if prec == "f64" else 4 + 8  # float working copy + double fallback copy
        assert ws >= 1003 * 1003 * es
    # chained triangular solves: a block counter, a timeout flag and one flag per 64-row block
    assert lib.genp_solve_workspace(100, 2, 0) >= (2 + 2) * 4
    assert lib.genp_solve_workspace(100, 2, 1) >= 100 * 2 * 4 + (2 + 2) * 4
    assert lib.genp_solve_workspace(100, 2, 4) >= 100 * 2 * 8
    assert lib.rbt_residual_workspace(1000, 3) >= 1000 * 3 * 8
    # the host-buffer solve: device copies of A, B and X in front of the solve's scratch
    o = _lib.make_opts(depth=2, prec="df64tc7", fallback=True)
    assert _lib.rbt_solve_host_workspace(o, 1003, 2) >= (_lib.rbt_solve_workspace(o, 1003, 2)
                                                         + 8 * 1003 * (1003 + 2 * 2))
    assert _lib.rbt_solve_host_workspace(_lib.make_opts(prec=9), 1003, 1) == 0      # invalid options


def test_host_solve_validates_without_gpu(lib):
    from paper_2312_09376_gb300 import _lib
    P = ctypes.c_void_p
    o = _lib.make_opts(depth=2, prec="df64tc7")
    info = _lib.rbt_info()
    args = (ctypes.byref(o), 10, 1)
    assert lib.rbt_solve_host(*args, P(8), 9, P(8), 10, P(8), 10, P(8), 1 << 30, ctypes.byref(info), None) == -1
    assert lib.rbt_solve_host(*args, None, 10, P(8), 10, P(8), 10, P(8), 1 << 30, ctypes.byref(info), None) == -1
    assert lib.rbt_solve_host(*args, P(8), 10, P(8), 10, P(8), 10, P(8), 16, ctypes.byref(info), None) == -3
    assert lib.rbt_solve_host(*args, P(8), 10, P(8), 10, P(8), 10, P(8), 1 << 30, None, None) == -1
    assert info.status == -1


def test_product_path_refuses_to_run_without_library(tmp_path, monkeypatch):
    from paper_2312_09376_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib._build, "build", lambda *a, **k: str(tmp_path / "missing.so"))
    with pytest.raises(Exception):
        _lib.load()


def test_rotation_gmres_entry_points_validate_on_host(lib):
    """The entry points of the rotation form and of the working-precision
    solve refuse bad arguments before any launch."""
    P = ctypes.c_void_p
    assert lib.rbt_generate_rot(-1, 2, 1, 1, None, None, 1, None) == -1
    assert lib.rbt_generate_rot(10, 2, -1, 1, P(8), P(8), 10, None) == -1      # align < 0
    assert lib.rbt_generate_rot(10, 2, 1, 1, P(8), P(8), 5, None) == -1        # ldw < n
    assert lib.rbt_generate_rot(10, 2, 1, 1, None, None, 10, None) == -1       # null pointers
    assert lib.rbt_generate_rot(0, 2, 1, 1, None, None, 1, None) == 0          # empty
    # unknown butterfly kind, unknown precision
    assert lib.rbt_transform_2sided(10, 2, 1, 7, 0, P(8), P(8), 10, P(8), 10, P(4096), 10, None) == -1
    assert lib.rbt_transform_2sided(10, 2, 1, 1, 9, P(8), P(8), 10, P(8), 10, P(4096), 10, None) == -1
    assert lib.rbt_transform_vec(10, 2, 1, 7, P(8), 10, 1, P(8), 10, 1, None) == -1
    assert lib.rbt_transform_vec(10, 2, 1, 1, P(8), 10, 1, P(8), 3, 1, None) == -1  # ldb < n
    # working-precision solve: bad precision, short workspace, empty
    assert lib.genp_solve_wp(10, 1, 7, P(8), 10, 0, P(8), 10, P(8), 1 << 20, None) == -1
    assert lib.genp_solve_wp(10, 1, 0, P(8), 10, 0, P(8), 10, P(8), 1, None) == -3
    assert lib.genp_solve_wp(0, 1, 0, None, 1, 0, None, 1, None, 0, None) == 0
    assert lib.genp_solve_wp_workspace(0, 1) == 0 and lib.genp_solve_wp_workspace(8, 0) == 0
    # the double-arithmetic solve keeps double inverses of the 64 x 64 diagonal blocks
    assert lib.genp_solve_wp_workspace(1000, 1) >= 16 * 64 * 64 * 8


def test_solve_options_validated(lib):
    from paper_2312_09376_gb300 import _lib
    assert _lib.rbt_solve_workspace(_lib.make_opts(kind="rotation"), 100, 1) > 0
    assert _lib.rbt_solve_workspace(_lib.make_opts(kind=5), 100, 1) == 0        # unknown kind
    assert _lib.rbt_solve_workspace(_lib.make_opts(refine="gmres", restart=65), 100, 1) == 0
    g = _lib.rbt_solve_workspace(_lib.make_opts(prec="f32", refine="gmres", restart=30), 1000, 1)
    s = _lib.rbt_solve_workspace(_lib.make_opts(prec="f32"), 1000, 1)
    assert g >= s + 31 * 1000 * 8        # the GMRES basis of 31 vectors comes on top


def test_wait_limit_and_stall_hooks_round_trip(lib):
    """The bounded-wait limit and the test stall are host settings read at
    launch time; setting them touches no GPU, and both restore their defaults."""
    from paper_2312_09376_gb300 import _lib
    default = _lib.rbt_debug_wait_limit(5_000_000)          # 5 ms
    assert default == 1_000_000_000                          # one second unless changed
    assert _lib.rbt_debug_wait_limit(0) == 5_000_000         # <= 0 restores the default
    assert _lib.rbt_debug_wait_limit(0) == 1_000_000_000
    assert _lib.rbt_debug_stall("chain") == 0
    assert _lib.rbt_debug_stall("oz_copy") == 1
    assert _lib.rbt_debug_stall(7) == 2                      # unknown values mean no stall
    assert _lib.rbt_debug_stall("none") == 0


def test_reference_size_query_matches_the_oracle():
    """rbt_reference_size (host) against the oracle's three rules: non-tiled,
    tiled, and the communication-free size of Eq. (comm-free-rbt-size)."""
    import oracle
    from paper_2312_09376_gb300 import _lib
    for n in (1, 2, 7, 1003, 20001, 40003):
        for d in (0, 1, 2, 3):
            assert _lib.rbt_reference_size(n, d) == oracle.ref_size(n, d)
            for nb in (16, 512):
                assert _lib.rbt_reference_size(n, d, nb) == oracle.ref_size(n, d, nb)
                for p, q in ((1, 1), (4, 4), (2, 3), (8, 1)):
                    assert _lib.rbt_reference_size(n, d, nb, (p, q)) == oracle.ref_size_comm_free(n, d, nb, p, q)
    assert _lib.rbt_reference_size(-1, 2) == -1
    assert _lib.rbt_reference_size(10, 2, 1, (4097, 1)) == -1
    assert _lib.rbt_reference_size(10, 2, 1 << 61, (4096, 4095)) == -1      # would overflow
    # an invalid grid makes the solve options invalid (size query 0)
    assert _lib.rbt_solve_workspace(_lib.make_opts(grid=(-1, 2)), 100, 1) == 0
    assert _lib.rbt_solve_workspace(_lib.make_opts(grid=(4, 4), align=64), 100, 1) > 0
