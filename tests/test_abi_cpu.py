"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every symbol the header declares, and the binding's constants match
the header."""
import ctypes
import os
import re

import pytest

import paper_1402_2518_gb300 as pkg
from paper_1402_2518_gb300 import linmin

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "linmin.h")


def _declared_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"LINMIN_API\s+[\w\s\*]+?\b(linmin_\w+)\s*\(", txt)))


def test_library_loads_and_exports_header_symbols():
    lib = pkg.load()
    declared = _declared_functions()
    assert declared, "no declarations found in include/linmin.h"
    for name in declared:
        assert hasattr(lib, name), f"{name} declared but not exported"
    assert sorted(linmin.EXPORTED) == declared


def test_no_other_exports():
    """Only the C ABI is visible (static CUDA runtime, hidden internals)."""
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", linmin.library_path()],
                         capture_output=True, text=True).stdout
    syms = [l.split()[-1] for l in out.splitlines() if " T " in l]
    assert sorted(syms) == sorted(linmin.EXPORTED), syms


def test_header_constants_match_binding():
    txt = open(HEADER).read()
    for name in ("LINMIN_STO", "LINMIN_SLO", "LINMIN_POS", "LINMIN_PROJ_DF", "LINMIN_PROJ_TC",
                 "LINMIN_PROJ_BF16"):
        m = re.search(rf"\b{name}\s*=\s*(\d+)", txt)
        assert m and int(m.group(1)) == getattr(linmin, name), name
    for name in ("LINMIN_OK", "LINMIN_ERR_INVALID", "LINMIN_ERR_OOM", "LINMIN_ERR_CUDA",
                 "LINMIN_ERR_RANK", "LINMIN_ERR_TIMEOUT", "LINMIN_ERR_NOT_CONVERGED",
                 "LINMIN_ERR_UNSUPPORTED"):
        m = re.search(rf"{name}\s*=\s*(\d+)", txt)
        assert m and int(m.group(1)) == getattr(linmin, name)
    for name in ("LINMIN_MAX_P", "LINMIN_MAX_L", "LINMIN_NOALLOC_SCRATCH_MB", "LINMIN_PHASE_RING",
                 "LINMIN_POS_SCALE"):
        m = re.search(rf"#define {name} (\d+)", txt)
        assert m and int(m.group(1)) == getattr(linmin, name)


def test_options_struct_layout_and_defaults():
    o = pkg.linmin_default_options()
    assert ctypes.sizeof(linmin.linmin_options) == 40
    assert o.max_iter == 100 and abs(o.tol - 1e-9) < 1e-15 and abs(o.refine_mu - 1e-9) < 1e-15
    assert o.precision == linmin.LINMIN_PROJ_TC and o.constraint == linmin.LINMIN_STO


def test_invalid_arguments_rejected_on_host():
    """Errors detected before any device work: no GPU is touched."""
    import numpy as np
    lib = pkg.load()
    h = ctypes.c_void_p()
    S = np.ones((4, 16), dtype=np.float32)
    assert lib.linmin_create(None, 16, 4, None, ctypes.byref(h)) == linmin.LINMIN_ERR_INVALID
    assert lib.linmin_create(S.ctypes.data_as(ctypes.c_void_p), 16, 0, None,
                             ctypes.byref(h)) == linmin.LINMIN_ERR_UNSUPPORTED
    assert lib.linmin_create(S.ctypes.data_as(ctypes.c_void_p), 16, linmin.LINMIN_MAX_P + 1,
                             None, ctypes.byref(h)) == linmin.LINMIN_ERR_UNSUPPORTED
    assert lib.linmin_create(S.ctypes.data_as(ctypes.c_void_p), 3, 4, None,
                             ctypes.byref(h)) == linmin.LINMIN_ERR_INVALID
    # four identical spectra: rank [S^T; 1^T] = 1 < 4
    assert lib.linmin_create(S.ctypes.data_as(ctypes.c_void_p), 16, 4, None,
                             ctypes.byref(h)) == linmin.LINMIN_ERR_RANK
    assert "rank" in pkg.linmin_last_error(None)
    bad = pkg.linmin_default_options()
    bad.max_iter = 0
    S2 = np.random.default_rng(0).uniform(0.2, 0.6, (4, 16)).astype(np.float32)
    assert lib.linmin_create(S2.ctypes.data_as(ctypes.c_void_p), 16, 4, ctypes.byref(bad),
                             ctypes.byref(h)) == linmin.LINMIN_ERR_INVALID
    assert lib.linmin_unmix(None, None, 0, None, None, None, None, None) == \
        linmin.LINMIN_ERR_INVALID
    # the batch call: no cubes, or a NULL handle in the list
    assert lib.linmin_unmix_batch(0, None, None, None, None, None, None, None, None) == \
        linmin.LINMIN_ERR_INVALID
    assert lib.linmin_unmix_batch(1, (ctypes.c_void_p * 1)(None), None, None, None, None, None,
                                  None, None) == linmin.LINMIN_ERR_INVALID
    assert lib.linmin_destroy(None) == linmin.LINMIN_OK


def test_binding_rejects_wrong_dtypes():
    import numpy as np
    with pytest.raises(TypeError):
        pkg.linmin_create(np.ones((4, 16)), 16, 4)          # float64
    with pytest.raises(ValueError):
        pkg.linmin_create(np.ones((16, 4), np.float32).T, 16, 4)  # not contiguous


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof/offsetof of every ABI struct, compiled from the header by the
    host C compiler, equal the ctypes layouts of the binding."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"linmin_options": linmin.linmin_options,
               "linmin_server_options": linmin.linmin_server_options,
               "linmin_request": linmin.linmin_request,
               "linmin_server_stats": linmin.linmin_server_stats,
               "linmin_detection": linmin.linmin_detection,
               "linmin_threshold_sums": linmin.linmin_threshold_sums}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "linmin.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append('return 0; }')
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(out[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)


def test_server_options_defaults_and_invalid():
    o = pkg.linmin_server_default_options()
    assert o.hbm_budget_bytes == 1 << 30 and o.slots == 4 and o.chunk_pixels == 65536
    assert o.max_iter == 100
    lib = pkg.load()
    bad = pkg.linmin_server_default_options()
    bad.slots = 0
    s = ctypes.c_void_p()
    assert lib.linmin_server_create(ctypes.byref(bad), ctypes.byref(s)) == linmin.LINMIN_ERR_INVALID
    assert lib.linmin_server_create(None, None) == linmin.LINMIN_ERR_INVALID
    assert lib.linmin_server_submit(None, None, None) == linmin.LINMIN_ERR_INVALID
    assert lib.linmin_server_destroy(None) == linmin.LINMIN_OK


def test_server_handle_bytes():
    b = pkg.linmin_server_handle_bytes(184, 36, 1000)
    b2 = pkg.linmin_server_handle_bytes(184, 36, 2000)
    bh = pkg.linmin_server_handle_bytes(184, 36, 1000, host_io=True)
    # per pixel: c~ hi/lo, x, lambda (4 P floats) + nu, iterations, retry,
    # mask, two lists, support size, pixel exponent (48 bytes); staging adds
    # cube + outputs
    assert b2 - b == 1000 * (16 * 36 + 48)
    assert bh - b == 1000 * (4 * 184 + 8 * 36 + 8) + 4 * 184
    assert pkg.linmin_server_handle_bytes(184, 65, 10) == 0


def test_lanes_entry_points_reject_null_handle():
    lib = pkg.load()
    assert lib.linmin_get_lanes(None) == -1
    assert lib.linmin_set_lanes(None, 4) == linmin.LINMIN_ERR_INVALID
    assert lib.linmin_autotune(None, None, 0, None, None, None, 0, None) == \
        linmin.LINMIN_ERR_INVALID


def test_constraint_rank_refusal_on_host():
    """slo / pos need rank S = P: the level/slope extras (0.5 flat - 0.5 u
    - 0.5 (1 - u) = 0, exact up to float32 rounding) are refused on the
    host, before any device work; sto accepts them."""
    import numpy as np
    import synth
    lib = pkg.load()
    cube = synth.make_cube(synth.OMEGA_262K, n_pix=1)
    h = ctypes.c_void_p()
    for c in (linmin.LINMIN_SLO, linmin.LINMIN_POS):
        opt = pkg.linmin_default_options()
        opt.constraint = c
        assert lib.linmin_create(cube.S.ctypes.data_as(ctypes.c_void_p), cube.L, cube.P,
                                 ctypes.byref(opt), ctypes.byref(h)) == linmin.LINMIN_ERR_RANK
    opt = pkg.linmin_default_options()
    opt.constraint = 7
    assert lib.linmin_create(cube.S.ctypes.data_as(ctypes.c_void_p), cube.L, cube.P,
                             ctypes.byref(opt), ctypes.byref(h)) == linmin.LINMIN_ERR_UNSUPPORTED


def test_noalloc_size_bound_on_host():
    """The scratch-size arithmetic of linmin_unmix_noalloc cannot wrap: N far
    beyond the array (up to 2^62, where a product N * (4P + 11) * 4 would
    overflow 64 bits) is refused, and the figure for a size that fits is
    consistent with the documented per-pixel cost.  Host arithmetic only."""
    st, b = pkg.linmin_noalloc_scratch_bytes(184, 36, 1 << 62)
    assert st == linmin.LINMIN_ERR_INVALID and b == 0
    st, b = pkg.linmin_noalloc_scratch_bytes(184, 32, (1 << 64) // (4 * (4 * 32 + 11)) + 1)
    assert st == linmin.LINMIN_ERR_INVALID
    st, b1 = pkg.linmin_noalloc_scratch_bytes(184, 36, 100000)
    st2, b2 = pkg.linmin_noalloc_scratch_bytes(184, 36, 100001)
    assert st == st2 == linmin.LINMIN_OK
    assert 4 * (4 * 36 + 11) <= b2 - b1 <= 4 * (4 * 36 + 11) + 11 * 256
    cap = linmin.LINMIN_NOALLOC_SCRATCH_MB << 20
    assert b1 <= cap
    # the largest N that fits, and the first that does not
    lo, hi = 1, cap
    while hi - lo > 1:
        mid = (lo + hi) // 2
        ok = pkg.linmin_noalloc_scratch_bytes(184, 36, mid)[0] == linmin.LINMIN_OK
        lo, hi = (mid, hi) if ok else (lo, mid)
    assert 100000 < lo < 110000
    assert pkg.linmin_noalloc_scratch_bytes(184, 36, hi)[0] == linmin.LINMIN_ERR_INVALID
    assert pkg.linmin_noalloc_scratch_bytes(184, 65, 10)[0] == linmin.LINMIN_ERR_UNSUPPORTED
    assert pkg.linmin_noalloc_scratch_bytes(184, 36, -1)[0] == linmin.LINMIN_ERR_INVALID
