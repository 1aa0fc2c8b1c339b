"""The C-ABI library loads and exports every entry point include/rt_api.h
declares; host-only entry points agree with the oracle (no GPU needed)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(rt_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    import ctypes
    import paper_2605_09882_gb300 as rt
    lib = ctypes.CDLL(rt.lib_path())
    names = _declared()
    assert len(names) >= 12, names
    for n in names:
        assert hasattr(lib, n), f"{n} declared but not exported"


def test_library_healpix_equals_oracle_bitwise():
    import oracle
    import paper_2605_09882_gb300 as rt
    for nside in (1, 2, 4, 8, 64):
        a = rt.healpix_dirs(nside)
        b = oracle.healpix(nside)
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), nside


def test_library_rejects_bad_nside():
    import paper_2605_09882_gb300 as rt
    for bad in (0, 3, 2048):
        with pytest.raises(rt.RTError):
            rt.healpix_dirs(bad)


def test_last_error_is_a_string():
    import paper_2605_09882_gb300 as rt
    assert isinstance(rt._lib.rt_last_error(), bytes)


def test_host_call_rejects_bad_arguments_before_any_device_work():
    import ctypes
    import paper_2605_09882_gb300 as rt
    lib = rt._lib
    buf = ctypes.create_string_buffer(4096)
    p = ctypes.cast(buf, ctypes.c_void_p)
    st = rt.Stats()

    def call(keys=p, levels=p, n=8, src=p, n_src=4, nside=1, dens=p, S=1, dt=0, mode=1, out=p, chunk=0):
        return lib.rt_trace_columns_host(keys, levels, n, None, src, n_src, nside, dens, S, dt, mode, out, chunk,
                                         ctypes.byref(st), None)

    ARG = 1
    assert call(keys=None) == ARG
    assert call(dens=None) == ARG
    assert call(src=None) == ARG and call(out=None) == ARG
    assert call(n=0) == ARG and call(n_src=-1) == ARG and call(chunk=-5) == ARG
    assert call(S=0) == ARG and call(S=9) == ARG
    assert call(dt=3) == ARG and call(mode=2) == ARG
    assert call(nside=0) == ARG
    assert b"rt_trace_columns_host" in lib.rt_last_error()
