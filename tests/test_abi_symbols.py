"""CPU checks of the C ABI boundary: the library builds, loads, and exports
every entry point declared in include/*.h (no compute calls: no GPU here)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(lqcd_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("lqcd_create", "lqcd_destroy", "lqcd_set_gauge", "lqcd_set_kappa", "lqcd_solve_batch",
                     "lqcd_loops_batch", "lqcd_noise_generate"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1108_2473_gb300 import build_lib, lqcd
    build_lib.build()
    lib = ctypes.CDLL(lqcd.LIB_PATH)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding names exactly the declared entry points
    assert set(lqcd.declared_symbols()) == _declared()


def test_binding_loads_and_reports_bad_arguments_without_gpu():
    from paper_1108_2473_gb300 import lqcd
    lib = lqcd.load()
    # argument validation happens before any device call
    rc = lib.lqcd_noise_generate(1, 0, 0, (ctypes.c_int * 4)(3, 4, 4, 4), 0, 0, 1, None, None)
    assert rc == lqcd.LQCD_ERR_INVALID
    assert "bad" in lqcd.lqcd_last_error(None)
    out = ctypes.c_void_p()
    assert lib.lqcd_create(ctypes.byref(out), (ctypes.c_int * 4)(4, 4, 5, 4), 0) == lqcd.LQCD_ERR_INVALID


def test_dilution_piece_count_matches_oracle_without_gpu():
    """lqcd_dilution_pieces is host-only: it agrees with the oracle's count for
    every base scheme with and without a spatial flag, and rejects bad input."""
    from oracle.philox import dilution_count, DIL_EO, DIL_CUBE
    from paper_1108_2473_gb300 import lqcd
    for dims in [(4, 4, 4, 8), (2, 2, 2, 4), (6, 4, 2, 10)]:
        for base in range(4):
            for sp in (0, DIL_EO, DIL_CUBE):
                assert lqcd.lqcd_dilution_pieces(dims, base | sp) == dilution_count(dims, base | sp)
    lib = lqcd.load()
    assert lib.lqcd_dilution_pieces((ctypes.c_int * 4)(4, 4, 4, 4), DIL_EO | DIL_CUBE) == -1
    assert lib.lqcd_dilution_pieces((ctypes.c_int * 4)(4, 3, 4, 4), 3) == -1
