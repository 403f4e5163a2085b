"""Host-only checks of the C ABI: the library loads, exports every entry point
that include/*.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2412_18271_b300 import mdpf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names |= set(re.findall(r"MDPF_API\s+[\w\s\*]*?\b(mdpf_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2412_18271_b300 import build
    build.build()
    return mdpf.load()


def test_header_declares_entry_points():
    names = declared_symbols()
    for required in ("mdpf_create", "mdpf_compute", "mdpf_step", "mdpf_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    # the Python binding marshals every declared entry point
    src = open(os.path.join(ROOT, "paper_2412_18271_b300", "mdpf.py")).read()
    missing = [n for n in declared_symbols() if '"%s"' % n not in src]
    assert not missing, missing


def _topo(n=3):
    el = np.zeros(n, dtype=np.int32)
    ms = np.ones(n)
    q = np.zeros(n)
    t = mdpf.mdpf_topology()
    t.n_atoms = n
    t.element = el.ctypes.data
    t.mass = ms.ctypes.data
    t.charge = q.ctypes.data
    t.n_bonds = 0
    return t, (el, ms, q)


@pytest.mark.parametrize("case", ["null_out", "zero_atoms", "bad_dt", "bad_mode", "bad_bond", "bad_mass",
                                  "bad_stepper", "bad_record_every", "learned_no_model", "learned_bad_magic",
                                  "learned_short", "learned_bad_alpha", "learned_bad_skin", "callback_no_provider"])
def test_create_rejects_bad_arguments_without_gpu(lib, case):
    t, keep = _topo()
    p = mdpf.mdpf_params()
    p.mode = mdpf.MDPF_MODE_PLAIN
    p.dt_fs = 0.5
    h = ctypes.c_void_p()
    out = ctypes.byref(h)
    expect = -1
    if case == "null_out":
        out = None
    elif case == "zero_atoms":
        t.n_atoms = 0
    elif case == "bad_dt":
        p.dt_fs = -1.0
    elif case == "bad_mode":
        p.mode = 7
    elif case == "learned_no_model":
        p.mode = mdpf.MDPF_MODE_LEARNED
    elif case in ("learned_bad_magic", "learned_short", "learned_bad_alpha"):
        from paper_2412_18271_b300 import model
        blob = bytearray(model.init_model(0).pack())
        if case == "learned_bad_magic":
            blob[0:8] = b"MDPFMLP2"
        elif case == "learned_short":
            blob = blob[:-4]
        else:
            blob[32:40] = np.array([0.2]).tobytes()
            expect = -8
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        keep = keep + (buf,)
        p.mode = mdpf.MDPF_MODE_LEARNED
        p.model = ctypes.addressof(buf)
        p.model_bytes = len(blob)
    elif case == "learned_bad_skin":
        p.mode = mdpf.MDPF_MODE_LEARNED
        p.skin = -1.0
    elif case == "callback_no_provider":
        p.mode = mdpf.MDPF_MODE_CALLBACK
    elif case == "bad_bond":
        b = np.array([[0, 5]], dtype=np.int32)
        r = np.array([1.0])
        keep = keep + (b, r)
        t.n_bonds = 1
        t.bonds = b.ctypes.data
        t.bond_r0 = r.ctypes.data
        t.bond_k = r.ctypes.data
    elif case == "bad_mass":
        keep[1][1] = 0.0
    elif case == "bad_stepper":
        p.stepper = 5
    elif case == "bad_record_every":
        p.energy_every = 3
        p.record_every = 10
        p.max_frames = 4
    rc = lib.mdpf_create(ctypes.byref(t), ctypes.byref(p), out)
    assert rc == expect
    assert not h.value
    assert len(lib.mdpf_last_error(None)) > 0


def test_null_context_is_rejected(lib):
    assert lib.mdpf_step(None, 1) == -1
    assert lib.mdpf_compute(None, None, None, None, None) == -1
    lib.mdpf_destroy(None)


@pytest.mark.parametrize("case", ["null", "n", "misaligned", "outside", "overlap"])
def test_tc_probe_rejects_bad_arguments(lib, case):
    # checked on the host before any CUDA call, so no device is needed
    fake = ctypes.c_void_p(256)
    n, a_off, b_off = 128, 0, 16384
    ptrs = [fake, fake, fake, fake]
    if case == "null":
        ptrs[2] = None
    elif case == "n":
        n = 96
    elif case == "misaligned":
        b_off = 16384 + 512
    elif case == "outside":
        b_off = 224 * 1024
    elif case == "overlap":
        b_off = 8192
    rc = lib.mdpf_debug_tc_probe(ptrs[0], ptrs[1], ptrs[2], n, a_off, b_off, ptrs[3], None)
    assert rc == -1   # MDPF_ERR_INVALID_ARG
    assert b"tc_probe" in lib.mdpf_last_error(None)
