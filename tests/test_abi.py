"""The C ABI library builds for sm_103a, loads, and exports every entry point that
include/dc.h declares; the ctypes layouts match the C structs (CPU only, no
compute calls)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dc.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2106_05306_gb300 import _lib, build
    build.build()
    return _lib.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dc_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dc_create_mesh", "dc_set_params", "dc_step", "dc_rollout", "dc_backward",
                     "dc_get_stats", "dc_sync", "dc_destroy", "dc_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2106_05306_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"{name} missing from the Python binding"


def test_struct_layouts_match_header(lib):
    from paper_2106_05306_gb300 import _lib
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "dc.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(dc_params), sizeof(dc_obstacle), sizeof(dc_stats),
         offsetof(dc_params, n_pd_iters), offsetof(dc_params, obstacles), offsetof(dc_stats, factor_nnz),
         offsetof(dc_stats, n_free), offsetof(dc_params, contact_compliance), offsetof(dc_params, adj_fallback),
         offsetof(dc_stats, adj_fallbacks), offsetof(dc_stats, device_bytes_peak));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "sz.c")
        exe = os.path.join(d, "sz")
        open(c, "w").write(prog)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(v) for v in subprocess.check_output([exe]).split()]
    P, O, S = _lib.dc_params, _lib.dc_obstacle, _lib.dc_stats
    want = [ctypes.sizeof(P), ctypes.sizeof(O), ctypes.sizeof(S), P.n_pd_iters.offset, P.obstacles.offset,
            S.factor_nnz.offset, S.n_free.offset, P.contact_compliance.offset, P.adj_fallback.offset,
            S.adj_fallbacks.offset, S.device_bytes_peak.offset]
    assert got == want


def test_default_params_and_error_path(lib):
    from paper_2106_05306_gb300 import _lib
    p = _lib.dc_params()
    lib.dc_default_params(ctypes.byref(p))
    assert p.n_pd_iters == 20 and abs(p.h - 1 / 120) < 1e-15 and p.gravity[1] == -9.8
    # host-side validation fails before any device work
    ctx = ctypes.c_void_p()
    st = lib.dc_create_mesh(ctypes.byref(ctx), 0, None, 0, None, 0, None, None)
    assert st == 1 and ctx.value is None
    assert b"null" in lib.dc_last_error(None)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2106_05306_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.replace("no CPU fallback", ""), f


def test_batch_hbm_bytes_runs_on_the_host(lib):
    """dc_batch_hbm_bytes orders, factorises and sizes on the host only (no device
    call), so it runs here: the footprint grows with the step count (one recorded
    state per step) and with the cloths, and invalid input is rejected."""
    import numpy as np
    import paper_2106_05306_gb300 as dc
    import scenes
    a, b = scenes.batch_instance(0), scenes.batch_instance(1)
    mesh = lambda s: (s.rest_pos, s.tris, s.pins)
    kw = dict(k_stretch=a.params.k_stretch, checkpoint_every=1)
    one = dc.batch_hbm_bytes([mesh(a)], kw, 10)
    assert one > 0
    assert dc.batch_hbm_bytes([mesh(a)], kw, 20) > one
    two = dc.batch_hbm_bytes([mesh(a), mesh(b)], kw, 10)
    assert two > one
    for bad in ([(a.rest_pos, np.array([[0, 1, 10 ** 6]]), [])], [mesh(a), mesh(b)]):
        with pytest.raises(dc.DCError):
            dc.batch_hbm_bytes(bad, [dict(kw), dict(kw, h=2e-2)] if len(bad) == 2 else kw, 10)


def test_every_mirrored_struct_matches_the_header_field_by_field(lib):
    """Every struct the binding mirrors (parameters, obstacles, statistics, batch
    instances, server configuration, requests, results, server statistics): its
    size and the offset of each of its fields, from the C compiler against the
    header, equal the ctypes mirror's."""
    from paper_2106_05306_gb300 import _lib
    structs = [_lib.dc_obstacle, _lib.dc_params, _lib.dc_stats, _lib.dc_instance, _lib.dc_server_config,
               _lib.dc_request, _lib.dc_result, _lib.dc_server_stats]
    lines, want = [], []
    for S in structs:
        name = S.__name__
        lines.append(f'  printf("%zu\\n", sizeof({name}));')
        want.append(ctypes.sizeof(S))
        for field in S._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({name}, {field[0]}));')
            want.append(getattr(S, field[0]).offset)
    prog = "#include <stdio.h>\n#include <stddef.h>\n#include \"dc.h\"\nint main(void) {\n" + "\n".join(lines) + \
        "\n  return 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "off.c")
        exe = os.path.join(d, "off")
        open(c, "w").write(prog)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(v) for v in subprocess.check_output([exe]).split()]
    assert got == want
