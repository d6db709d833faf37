"""C-ABI checks that need no GPU: libcofem builds/loads, exports every entry
point declared in include/*.h, and rejects bad arguments before touching a device."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DECL = re.compile(r"^\s*(?:cofem_status|void|const char\s*\*|long long)\s+(cofem_\w+)\s*\(", re.M)


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        names |= set(DECL.findall(open(h).read()))
    return sorted(names)


@pytest.fixture(scope="module")
def cf():
    lib = os.path.join(ROOT, "paper_2105_10439_gb300", "libcofem.so")
    if not os.path.exists(lib):
        import __graft_entry__
        __graft_entry__.build()
    import paper_2105_10439_gb300 as m
    return m


def test_header_declares_entry_points():
    names = _declared()
    for n in ("cofem_create", "cofem_fit", "cofem_destroy", "cofem_status_string",
              "cofem_probe_fill", "cofem_apply_operator"):
        assert n in names


def test_library_exports_every_declared_symbol(cf):
    lib = ctypes.CDLL(cf.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_binding(cf, tmp_path):
    """Every field of the ABI structs sits at the same offset, and every struct
    has the same size, in the C header (compiled here with the host C compiler)
    as in the ctypes binding."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"cofem_opts": cf.cofem_opts, "cofem_request": cf.cofem_request, "cofem_result": cf.cofem_result,
               "cofem_server_stats": cf.cofem_server_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cofem.h"', "int main(void) {"]
    for sname, cls in structs.items():
        lines.append(f'    printf("{sname} size %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{sname} {fname} %zu\\n", offsetof({sname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        a, b, v = ln.split()
        got[(a, b)] = int(v)
    for sname, cls in structs.items():
        assert got[(sname, "size")] == ctypes.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert got[(sname, fname)] == getattr(cls, fname).offset, (sname, fname)


def test_status_strings_and_defaults(cf):
    assert cf.lib.cofem_status_string(0) == b"ok"
    assert cf.lib.cofem_status_string(1) == b"invalid argument"
    o = cf.default_opts()
    assert o.precision == cf.COFEM_F32 and o.alpha_max == 1e12 and o.use_graph == 1 and o.seed == 2
    # the remaining defaults as the header documents them
    assert (o.precond, o.conv, o.rr_period, o.stream) == (cf.COFEM_PRECOND_JACOBI, cf.COFEM_CONV_PER_COLUMN, 0, None)
    assert (o.dense_path, o.max_sms, o.overlap_launch, o.prior) == (cf.COFEM_PATH_AUTO, 0, 1, cf.COFEM_PRIOR_GAUSSIAN)
    assert o.check_residual == 0 and o.warm_start == 0 and o.toeplitz_path == 0
    assert o.residual_path == cf.COFEM_RESIDUAL_AUTO


@pytest.mark.parametrize("args,msg", [
    ((0, 4, 0, 0), "bad N/D"),
    ((4, -1, 0, 0), "bad N/D"),
    ((4, 4, 7, 0), "unknown dictionary kind"),
    ((4, 4, 0, 3), "L must be 0"),
    ((4, 5, 1, 2), "N == D"),
    ((8, 8, 1, 0), "1 <= L"),
    ((8, 8, 1, 2000), "1 <= L"),
])
def test_create_rejects_bad_arguments_without_gpu(cf, args, msg):
    N, D, kind, L = args
    with pytest.raises(cf.CofemError) as e:
        cf.cofem_create(N, D, kind, np.zeros(64, np.float32), L, cf.default_opts())
    assert e.value.status == cf.COFEM_ERR_INVALID_ARG
    assert msg in str(e.value)


def test_create_rejects_bad_opts(cf):
    for kw in (dict(precision=9), dict(precond=4), dict(conv=3), dict(rr_period=-1), dict(alpha_max=-1.0),
               dict(max_sms=-1), dict(dense_path=7), dict(overlap_launch=2), dict(prior=5),
               dict(check_residual=2), dict(warm_start=3), dict(residual_path=3), dict(residual_path=-1)):
        with pytest.raises(cf.CofemError) as e:
            cf.cofem_create(4, 4, 0, np.zeros(16, np.float32), 0, cf.default_opts(**kw))
        assert e.value.status == cf.COFEM_ERR_INVALID_ARG


def test_null_handle_calls(cf):
    with pytest.raises(cf.CofemError) as e:
        cf.cofem_fit(None, np.zeros(4, np.float32), 1.0, None, 2, 2, 1e-5, 10,
                     np.zeros(4, np.float32), np.zeros(4, np.float32), np.zeros(4, np.float32))
    assert e.value.status == cf.COFEM_ERR_INVALID_ARG
    cf.cofem_destroy(None)   # accepted
    with pytest.raises(cf.CofemError) as e:
        cf.cofem_true_residuals(None, 2, 3)
    assert e.value.status == cf.COFEM_ERR_INVALID_ARG
    x = np.zeros((2, 4), np.float32)
    with pytest.raises(cf.CofemError) as e:
        cf.cofem_accurate_product(None, x, x, 2, np.zeros((2, 4), np.float64))
    assert e.value.status == cf.COFEM_ERR_INVALID_ARG


def test_probe_fill_rejects_bad_sizes(cf):
    with pytest.raises(cf.CofemError):
        cf.cofem_probe_fill(1, 1, 0, 10, np.zeros(10, np.float32))
