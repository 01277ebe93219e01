"""The C-ABI library loads on a machine without a GPU and exports every symbol
that include/isg.h declares; argument checks that need no device answer with
status codes."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "isg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(isg_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def isg():
    from paper_1411_0127_gb300 import build
    build.build()
    import paper_1411_0127_gb300 as m
    m.lib()
    return m


def test_every_declared_symbol_is_exported_and_bound(isg):
    names = declared_functions()
    assert len(names) >= 18
    lib = ctypes.CDLL(isg.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), "libisg.so does not export %s" % n
        assert n in isg.SIGNATURES, "binding lacks %s" % n
    assert set(isg.SIGNATURES) == set(names)


def test_create_rejects_bad_arguments_without_touching_the_device(isg):
    h = ctypes.c_void_p()
    lib = isg.lib()
    for L, beta, kind in [(5, 1.0, 0), (2, 1.0, 0), (2050, 1.0, 0), (8, 0.0, 0), (8, -2.0, 0),
                          (8, float("nan"), 0), (8, 1.0, 7)]:
        rc = lib.isg_create(L, 1, 2, beta, kind, ctypes.byref(h))
        assert rc == isg.ISG_ERR_ARG
        assert h.value is None
        assert lib.isg_last_error()
    assert lib.isg_create(8, 1, 2, 1.0, 0, None) == isg.ISG_ERR_ARG


def test_amsc_create_rejects_bad_arguments_without_touching_the_device(isg):
    h = ctypes.c_void_p()
    lib = isg.lib()
    seeds = (ctypes.c_uint64 * 32)(*range(32))
    for L, beta, kind in [(5, 1.0, 0), (2, 1.0, 0), (1026, 1.0, 0), (8, 0.0, 0), (8, -1.0, 1),
                          (8, float("nan"), 0), (8, 1.0, 3)]:
        assert lib.isg_amsc_create(L, seeds, seeds, 3, beta, kind, ctypes.byref(h)) == isg.ISG_ERR_ARG
        assert h.value is None
    assert lib.isg_amsc_create(8, None, seeds, 3, 1.0, 0, ctypes.byref(h)) == isg.ISG_ERR_ARG
    assert lib.isg_amsc_create(8, seeds, seeds, 3, 1.0, 0, None) == isg.ISG_ERR_ARG
    assert lib.isg_amsc_sweep(None, 1, None) == isg.ISG_ERR_ARG
    assert lib.isg_amsc_energies(None, None, None) == isg.ISG_ERR_ARG
    assert lib.isg_amsc_read_spins(None, 0, None, 0, None) == isg.ISG_ERR_ARG
    with pytest.raises(ValueError):
        isg.Amsc(8, [1] * 31, [2] * 32, 3, 1.0, "minstd")


def test_other_host_side_checks(isg):
    lib = isg.lib()
    assert lib.isg_read_spins_packed(None, None, 0, None) == isg.ISG_ERR_ARG
    assert lib.isg_exchange_async(None, None, None, 0, 1, None, None) == isg.ISG_ERR_ARG
    assert lib.isg_batch_set_config(None, 0, 0, 1, 1) == isg.ISG_ERR_ARG
    assert lib.isg_int_rate(3, None) == isg.ISG_ERR_ARG
    assert lib.isg_batch_get_config(None, None, None, None, None) == isg.ISG_ERR_ARG
    assert lib.isg_write_spins_packed(None, None, 0, None) == isg.ISG_ERR_ARG
    assert lib.isg_info(None, None, None, None, None, None) == isg.ISG_ERR_ARG
    assert lib.isg_sweep(None, 1, None) == isg.ISG_ERR_ARG
    assert lib.isg_sweep_test_stall(None) == isg.ISG_ERR_ARG
    assert lib.isg_sweep_info(None, None) == isg.ISG_ERR_ARG
    # one allocator function without the other
    f = isg._ALLOC_T(lambda n, c: None)
    assert lib.isg_set_allocator(ctypes.cast(f, ctypes.c_void_p), None, None) == isg.ISG_ERR_ARG
    assert lib.isg_set_allocator(None, None, None) == isg.ISG_OK
    # a buffer that is not a checkpoint
    h = ctypes.c_void_p()
    junk = ctypes.create_string_buffer(b"not a checkpoint" * 16)
    assert lib.isg_load(junk, 256, ctypes.byref(h)) == isg.ISG_ERR_ARG
    assert lib.isg_load(junk, 3, ctypes.byref(h)) == isg.ISG_ERR_ARG
    assert b"checkpoint" in lib.isg_last_error() or b"truncated" in lib.isg_last_error()


def test_allocation_failure_is_reported(isg):
    """An allocator that refuses: isg_create returns ISG_ERR_NOMEM, frees what it
    got and touches no device (runs without a GPU)."""
    lib = isg.lib()
    calls = {"alloc": 0, "free": 0}

    def refuse(size, ctx):
        calls["alloc"] += 1
        return None

    def release(ptr, ctx):
        calls["free"] += 1

    a, f = isg._ALLOC_T(refuse), isg._FREE_T(release)
    assert lib.isg_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None) == isg.ISG_OK
    try:
        h = ctypes.c_void_p()
        rc = lib.isg_create(64, 1, 2, 1.0, isg.ISG_RNG_MT19937, ctypes.byref(h))
        assert rc == isg.ISG_ERR_NOMEM
        assert h.value is None
        assert b"allocation failed" in lib.isg_last_error()
        assert calls["alloc"] >= 1 and calls["free"] == 0   # nothing was obtained, nothing to free
    finally:
        assert lib.isg_set_allocator(None, None, None) == isg.ISG_OK


def test_binding_raises_with_message(isg):
    with pytest.raises(isg.IsgError) as ei:
        isg.Sim(7, 1, 2, 1.0, "minstd")
    assert ei.value.code == isg.ISG_ERR_ARG
    assert "L=7" in str(ei.value)
