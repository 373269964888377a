"""The C-ABI library builds, loads and exports every entry point include/rtcur.h declares, and
rejects invalid arguments before touching a GPU (CPU only)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_2108_10448_gb300 import rtcur as rt
    return rt.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "rtcur.h")).read()
    return sorted(set(re.findall(r"RTCUR_API\s+[\w\s\*]+?\b(rtcur_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("kw,msg", [
    (dict(dims=[10, 10, 10, 10, 10]), "n_modes"),
    (dict(gamma=1.0), "gamma"),
    (dict(gamma=0.0), "gamma"),
    (dict(tol=float("nan")), "tol"),
    (dict(max_iter=0), "max_iter"),
    (dict(variant=2), "variant"),
    (dict(ranks=[0, 2, 2]), "ranks"),
    (dict(nI=[1, 4, 4]), "nI"),
    (dict(nI=[11, 4, 4]), "nI"),
    (dict(nJ=[101, 8, 8]), "nJ"),
])
def test_create_rejects_invalid_arguments(lib, kw, msg):
    from paper_2108_10448_gb300 import rtcur as rt
    args = dict(dims=[10, 10, 10], ranks=[2, 2, 2], nI=[4, 4, 4], nJ=[8, 8, 8], zeta0=1.0,
                gamma=0.7, tol=1e-5, max_iter=10, variant=0)
    args.update(kw)
    n = len(args["dims"])
    for key in ("ranks", "nI", "nJ"):
        if len(args[key]) < n:
            args[key] = list(args[key]) + [args[key][-1]] * (n - len(args[key]))
    with pytest.raises(rt.RTCURError) as ei:
        rt.rtcur_create(**args)
    assert ei.value.status == rt.EINVAL
    assert msg in str(ei.value)


def test_options_reserved_must_be_zero(lib):
    from paper_2108_10448_gb300 import rtcur as rt
    o = rt.make_options()
    o.reserved[1] = 1
    with pytest.raises(rt.RTCURError) as ei:
        rt.rtcur_create([8, 8, 8], [2, 2, 2], [4, 4, 4], [8, 8, 8], 1.0, 0.7, 1e-5, 5, 0, o)
    assert ei.value.status == rt.EINVAL


def test_checkpoint_options_are_validated(lib):
    from paper_2108_10448_gb300 import rtcur as rt
    for dims, ck, msg in (([8, 8, 8], 6, "checkpoint must be in"),
                          ([8, 8, 8, 8], 2, "n_modes == 3")):
        n = len(dims)
        with pytest.raises(rt.RTCURError) as ei:
            rt.rtcur_create(dims, [2] * n, [4] * n, [8] * n, 1.0, 0.7, 1e-5, 5, 0,
                            rt.make_options(checkpoint=ck))
        assert ei.value.status == rt.EINVAL
        assert msg in str(ei.value)


def test_s_format_options_are_validated(lib):
    from paper_2108_10448_gb300 import rtcur as rt
    for dims, kw, msg in (([8, 8, 8], dict(s_format=2), "s_format must be"),
                          ([8, 8, 8], dict(s_format=rt.S_COMPRESSED), "needs the FULL scope"),
                          ([8, 8, 8], dict(s_format=rt.S_COMPRESSED, scope=rt.SCOPE_FULL,
                                           dense_form=rt.FORM_BF16), "dense_form FP32"),
                          ([8, 8, 10], dict(s_format=rt.S_COMPRESSED, scope=rt.SCOPE_FULL), "d_n % 4 == 0")):
        with pytest.raises(rt.RTCURError) as ei:
            rt.rtcur_create(dims, [2, 2, 2], [4, 4, 4], [8, 8, 8], 1.0, 0.7, 1e-5, 5, 0, rt.make_options(**kw))
        assert ei.value.status == rt.EINVAL
        assert msg in str(ei.value)


def test_compressed_s_geometry_is_validated(lib):
    from paper_2108_10448_gb300 import rtcur as rt
    o = rt.make_options(scope=rt.SCOPE_FULL, s_format=rt.S_COMPRESSED)
    for dims, ranks, nI, nJ in (([4, 4, 4100], [2, 2, 2], [4, 4, 4], [8, 8, 8]),   # d_n > 4096
                                ([20, 20, 40], [2, 2, 9], [4, 4, 12], [8, 8, 20])):  # r_n > 8
        with pytest.raises(rt.RTCURError) as ei:
            rt.rtcur_create(dims, ranks, nI, nJ, 1.0, 0.7, 1e-5, 5, 0, o)
        assert ei.value.status == rt.EINVAL
        assert "s_format COMPRESSED needs d_n % 4 == 0" in str(ei.value)


def test_compressed_s_calls_reject_a_null_plan(lib):
    import ctypes as C
    from paper_2108_10448_gb300 import rtcur as rt
    out = rt.rtcur_s_compressed()
    assert lib.rtcur_get_s_compressed(None, C.byref(out), None) == rt.EINVAL
    assert lib.rtcur_compact_s(None, None, None, None) == rt.EINVAL
    assert lib.rtcur_decode_s(None, None, None) == rt.EINVAL


def test_header_compiles_as_c_and_matches_the_binding(tmp_path):
    # the boundary is plain C: the header compiles as C99, and its structs have the layout the
    # ctypes binding declares (sizes and field offsets)
    import ctypes as C
    import shutil
    import subprocess
    from paper_2108_10448_gb300 import rtcur as rt
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"rtcur_options": rt.rtcur_options, "rtcur_result": rt.rtcur_result,
               "rtcur_s_compressed": rt.rtcur_s_compressed}
    lines = ['#include "rtcur.h"', "#include <stddef.h>", "#include <stdio.h>", "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                  text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"
