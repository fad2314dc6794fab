"""The C-ABI library builds, loads, exports every declared symbol and rejects bad arguments
before touching the GPU (no compute calls: these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dopinf.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    path = g.build()
    return ctypes.CDLL(path)


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dopinf_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 10
    for s in syms:
        assert hasattr(lib, s), s
    from paper_2504_14338_gb300 import build as b
    out = subprocess.run(["nm", "-D", "--defined-only", b.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dopinf_\w+)", out))
    assert set(syms) <= exported
    assert all(e in syms for e in exported), "exported symbols not declared in dopinf.h"


def test_status_strings(lib):
    lib.dopinf_status_string.restype = ctypes.c_char_p
    assert lib.dopinf_status_string(0) == b"ok"
    assert b"argument" in lib.dopinf_status_string(-1)


def test_arguments_rejected_before_launch():
    from paper_2504_14338_gb300 import dopinf as dp
    L = dp.lib
    offs = (ctypes.c_int64 * 3)(0, 5, 10)
    z = ctypes.c_void_p(0)
    # k = 0, bad offsets, too many variables, missing workspace
    assert L.dopinf_transform(z, 0, 10, 0, 10, 2, offs, 3, z, z, z, z, 0, z) == dp.E_ARG
    bad = (ctypes.c_int64 * 3)(0, 7, 9)
    assert L.dopinf_transform(ctypes.c_void_p(8), 0, 10, 4, 10, 2, bad, 3, ctypes.c_void_p(8),
                              ctypes.c_void_p(8), z, z, 0, z) == dp.E_ARG
    assert L.dopinf_transform(ctypes.c_void_p(8), 2, 10, 4, 10, 2, offs, 3, ctypes.c_void_p(8),
                              ctypes.c_void_p(8), z, z, 0, z) == dp.E_ARG
    assert L.dopinf_transform(ctypes.c_void_p(8), 0, 10, 4, 10, 2, offs, 3, ctypes.c_void_p(8),
                              ctypes.c_void_p(8), z, z, 0, z) == dp.E_ARG      # no flags word, no ws
    assert L.dopinf_transform(ctypes.c_void_p(8), 0, 10, 4, 5, 2, offs, 3, ctypes.c_void_p(8),
                              ctypes.c_void_p(8), ctypes.c_void_p(8), z, 0, z) == dp.E_ARG  # ldq < n
    # Gram: ldq < n, unknown mode, ldd < k
    assert L.dopinf_gram(ctypes.c_void_p(8), 0, 100, 4, 50, 0, 0, ctypes.c_void_p(8), 4, z, 0, z) == dp.E_ARG
    assert L.dopinf_gram(ctypes.c_void_p(8), 0, 100, 4, 100, 7, 0, ctypes.c_void_p(8), 4, z, 0, z) == dp.E_UNSUPPORTED
    assert L.dopinf_gram(ctypes.c_void_p(8), 0, 100, 4, 100, 0, 0, ctypes.c_void_p(8), 3, z, 0, z) == dp.E_ARG
    # reduce: r_cap > k, r_fixed > r_cap, energy target out of range
    r = ctypes.c_int(0)
    t = ctypes.c_double(0)
    p8 = ctypes.c_void_p(8)
    assert L.dopinf_reduce(p8, 5, 5, 0.99, 0, 6, ctypes.byref(r), ctypes.byref(t), p8, p8, p8, z, 0, z) == dp.E_ARG
    assert L.dopinf_reduce(p8, 5, 5, 0.99, 4, 3, ctypes.byref(r), ctypes.byref(t), p8, p8, p8, z, 0, z) == dp.E_ARG
    assert L.dopinf_reduce(p8, 5, 5, 1.5, 0, 3, ctypes.byref(r), ctypes.byref(t), p8, p8, p8, z, 0, z) == dp.E_ARG
    # learn: n_steps < k, r > r_max
    rl = (ctypes.c_int * 1)(3)
    b = (ctypes.c_double * 1)(1e-3)
    best = ctypes.c_int(0)
    assert L.dopinf_learn(p8, 3, 50, 3, rl, 1, b, 1, b, 1, 0, 1.0, 10, 1.2, p8, p8, p8, z, ctypes.byref(best), p8,
                          None, p8, 1 << 30, z) == dp.E_ARG
    rl4 = (ctypes.c_int * 1)(4)
    assert L.dopinf_learn(p8, 3, 50, 3, rl4, 1, b, 1, b, 1, 0, 1.0, 100, 1.2, p8, p8, p8, z, ctypes.byref(best), p8,
                          None, p8, 1 << 30, z) == dp.E_ARG
    # allocation-free Gram: k beyond its fixed array is refused before any tile count or CUDA call
    f = L.dopinf_gram_fp64_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    for k in (2817, 5_000_000, 1 << 40):
        assert f(p8, 0, 64, k, 64, 0, p8, k, z) == dp.E_UNSUPPORTED, k
    assert f(p8, 0, 64, 100, 63, 0, p8, 100, z) == dp.E_ARG      # ldq < n
    # rollout: r = 0, ldo < r; r = 93 is past the widest kernel
    assert L.dopinf_rollout(p8, 93, 93, p8, 10, 0, 1.0, p8, p8, z) == dp.E_UNSUPPORTED
    assert L.dopinf_rollout(p8, 0, 1, p8, 10, 0, 1.0, p8, p8, z) == dp.E_ARG
    assert L.dopinf_rollout(p8, 3, 2, p8, 10, 0, 1.0, p8, p8, z) == dp.E_ARG


def test_workspace_queries_are_host_only_and_monotone():
    from paper_2504_14338_gb300 import dopinf as dp
    L = dp.lib
    g1 = L.dopinf_gram_workspace(10_000, 200, 0, 0)
    g2 = L.dopinf_gram_workspace(10_000, 600, 0, 0)
    assert 0 < g1 < g2 and g1 % 256 == 0
    assert L.dopinf_reduce_workspace(600, 30) > L.dopinf_reduce_workspace(200, 30) > 0
    rl = (ctypes.c_int * 3)(10, 20, 30)
    assert L.dopinf_learn_workspace(30, 600, rl, 3, 8, 8) > L.dopinf_learn_workspace(30, 600, rl, 1, 8, 8) > 0
