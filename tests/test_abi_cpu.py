"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every entry point that include/acom.h declares, and rejects invalid
arguments before touching the device."""

import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "acom.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2111_00171_gb300 import acom
    return acom.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(acom_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("acom_plan_create", "acom_match", "acom_plan_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2111_00171_gb300 import acom
    names = declared_functions()
    for n in names:
        assert hasattr(lib, n), n
    assert set(acom.EXPORTED) <= set(names)
    assert lib.acom_version() >= 1


def test_status_strings(lib):
    for code, name in [(0, b"ACOM_OK"), (1, b"ACOM_ERR_INVALID_ARG"), (6, b"ACOM_ERR_BAD_INPUT")]:
        assert lib.acom_status_str(code) == name


def _args(n_phi=180, step=2.0, n_atoms=4, delta=0.08):
    from paper_2111_00171_gb300 import acom
    cr = acom.Crystal()
    for i in range(3):
        cr.lattice[i][i] = 4.08
    pos = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], dtype=np.float64)
    ff = np.full(4, 79.0)
    fb = np.full(4, 0.25)
    dp = C.POINTER(C.c_double)
    cr.n_atoms = n_atoms
    cr.frac_pos = pos.ctypes.data_as(dp)
    cr.ff_A = ff.ctypes.data_as(dp)
    cr.ff_B = fb.ctypes.data_as(dp)
    g = acom.ZaGrid()
    for i, v in enumerate([[0, 0, 1], [0, 1, 1], [1, 1, 1]]):
        for j in range(3):
            g.v[i][j] = v[j]
    g.step_deg = step
    g.solid_angle = 4 * np.pi / 48
    sh = acom.Shells(75, 0.02)
    op = acom.PlanOpts(delta, 1.0, 1.0, 0.01969, 1.5, 0)
    keep = (pos, ff, fb)
    return cr, g, sh, n_phi, op, keep


@pytest.mark.parametrize("bad", ["odd_nphi", "big_nphi", "step0", "atoms0", "delta0"])
def test_plan_create_rejects_invalid_arguments(lib, bad):
    kw = {"odd_nphi": dict(n_phi=181), "big_nphi": dict(n_phi=2048), "step0": dict(step=0.0),
          "atoms0": dict(n_atoms=0), "delta0": dict(delta=0.0)}[bad]
    cr, g, sh, n_phi, op, keep = _args(**kw)
    h = C.c_void_p()
    st = lib.acom_plan_create(C.byref(cr), C.byref(g), C.byref(sh), n_phi, 0.02, C.byref(op),
                              None, C.byref(h))
    assert st == 1, lib.acom_last_error()
    assert not h.value
    assert lib.acom_last_error()


def test_match_rejects_null_plan(lib):
    from paper_2111_00171_gb300 import acom
    pk = acom.PeaksCSR(0, None, None, None, None)
    res = acom.Result()
    assert lib.acom_match(None, C.byref(pk), None, C.byref(res), None) == 1


def test_concat_rejects_invalid_arguments_on_host(lib):
    """acom_plan_concat and acom_plan_get_phases check their arguments before
    any device work."""
    h = C.c_void_p()
    assert lib.acom_plan_concat(None, 1, None, C.byref(h)) == 1
    arr = (C.c_void_p * 1)(None)
    assert lib.acom_plan_concat(arr, 0, None, C.byref(h)) == 1
    assert lib.acom_plan_concat(arr, 1, None, C.byref(h)) == 1     # a null plan
    assert lib.acom_plan_concat(arr, 1, None, None) == 1
    assert not h.value
    out = (C.c_int32 * 2)()
    assert lib.acom_plan_get_phases(None, out) == 1


def test_refine_defaults_and_argument_checks_on_host(lib):
    """acom_refine_defaults is host-only; acom_refine and
    acom_kinematical_score reject a null plan before any device work."""
    from paper_2111_00171_gb300 import acom
    d = lib.acom_refine_defaults()
    assert (d.steps, d.twin) == (20, 1)
    assert (d.rho_start, d.rho_end, d.damping, d.max_step_deg) == pytest.approx((0.15, 0.03, 0.3, 1.0))
    pk = acom.PeaksCSR(0, None, None, None, None)
    assert lib.acom_refine(None, C.byref(pk), None, None, None, None, None, None) == 1
    assert lib.acom_kinematical_score(None, C.byref(pk), None, None, 0.03, None, None, None,
                                      None) == 1


def _header_struct_fields(name):
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + ";", text).group(1)
    return re.findall(r"\b([a-z_][a-z_0-9]*)\s*;", body)


def test_autotune_and_tile_order_argument_checks_on_host(lib):
    """acom_autotune rejects a null plan or result before any device work; the
    ctypes mirrors of acom_match_opts and acom_tune_result carry the header's
    fields in the header's order (every field 32 bits wide)."""
    from paper_2111_00171_gb300 import acom
    pk = acom.PeaksCSR(0, None, None, None, None)
    best = acom.TuneResult()
    assert lib.acom_autotune(None, C.byref(pk), None, C.byref(best), None, None) == 1
    assert lib.acom_last_error()
    for mirror, name in ((acom.MatchOpts, "acom_match_opts"), (acom.TuneResult, "acom_tune_result")):
        fields = _header_struct_fields(name)
        assert [f for f, _ in mirror._fields_] == fields, name
        assert C.sizeof(mirror) == 4 * len(fields), name
