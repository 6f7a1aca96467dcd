"""The C-ABI library on the host (no GPU compute): it loads, exports every symbol
that include/stg.h declares, and its host-side logic (geometry, sizes, argument
validation) behaves as documented."""
import ctypes
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1801_01473_gb300 import build as b
    b.build()
    from paper_1801_01473_gb300.lib import lib
    return lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "stg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(stg_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = declared_symbols()
    assert len(names) >= 19
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    from paper_1801_01473_gb300.lib import EXPORTS
    assert sorted(EXPORTS) == names


def _lat(L, dims, ap=1):
    h = ctypes.c_void_p()
    rc = L.stg_lattice_create((ctypes.c_int32 * 4)(*dims), ap, ctypes.byref(h))
    return rc, h


def test_lattice_geometry_and_sizes(L):
    rc, h = _lat(L, (6, 4, 2, 8))
    assert rc == 0
    assert L.stg_lattice_sites(h, -1) == 384
    assert L.stg_lattice_sites(h, 0) == 192 and L.stg_lattice_sites(h, 1) == 192
    assert L.stg_lattice_sites(h, 2) == -1
    sizes = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_sizes.json")))
    # FP64 pseudofermion: 3 double complex = 48 bytes per site (Sec. 3.1)
    assert L.stg_field_bytes(h, 0) == 192 * sizes["fermion_bytes_per_site_fp64"]["value"]
    assert L.stg_field_bytes(h, 1) == 192 * 24
    assert L.stg_field_bytes(h, 4) == 192 * 48  # double-single: two floats per real
    assert L.stg_field_bytes(h, 2) == 0
    L.stg_lattice_destroy(h)


@pytest.mark.parametrize("dims", [(3, 4, 4, 4), (4, 4, 4, 5), (0, 4, 4, 4), (4, 4, 4, -2)])
def test_lattice_rejects_bad_extents(L, dims):
    rc, h = _lat(L, dims)
    assert rc == -2 and not h.value
    assert b"even" in L.stg_last_error()


def test_null_arguments_rejected_before_launch(L):
    rc, h = _lat(L, (4, 4, 4, 4))
    out = ctypes.c_void_p()
    assert L.stg_lattice_create(None, 1, ctypes.byref(out)) == -1
    assert L.stg_gauge_create(h, None, 0, 18, None, ctypes.byref(out)) == -1
    assert L.stg_gauge_create(None, ctypes.c_void_p(256), 0, 18, None, ctypes.byref(out)) == -1
    # bad precision/compression pairs: 16-bit links need 12-real compression
    assert L.stg_gauge_create(h, ctypes.c_void_p(256), 2, 18, None, ctypes.byref(out)) == -1
    assert L.stg_gauge_create(h, ctypes.c_void_p(256), 7, 18, None, ctypes.byref(out)) == -1
    assert L.stg_gauge_create(h, ctypes.c_void_p(256), 0, 11, None, ctypes.byref(out)) == -1
    # misaligned pointer
    assert L.stg_gauge_create(h, ctypes.c_void_p(8), 0, 18, None, ctypes.byref(out)) == -1
    assert L.stg_dslash_eo(None, ctypes.c_void_p(256), ctypes.c_void_p(512), None) == -1
    assert L.stg_field_pack(h, 2, ctypes.c_void_p(256), ctypes.c_void_p(512), None) == -1
    assert L.stg_fermion_force(None, 1, None, None, None, 0, None) == -1
    assert L.stg_mscg_solve(None, None, None, None, None, None, None) == -1
    assert L.stg_mscg_solve_batched(0, None, None, None) == -1
    L.stg_lattice_destroy(h)


def test_stout_arguments_rejected_before_launch(L):
    rc, h = _lat(L, (4, 4, 4, 4))
    a, b, c, d = (ctypes.c_void_p(v) for v in (256, 512, 768, 1024))
    smear, force = L.stg_stout_smear, L.stg_stout_force
    assert smear(None, 0, 1, 0.1, a, b, None) == -1
    assert smear(h, 0, 0, 0.1, a, b, None) == -1 and b"nstep" in L.stg_last_error()
    assert smear(h, 0, 17, 0.1, a, b, None) == -1
    assert smear(h, 0, 1, 0.6, a, b, None) == -1 and b"rho" in L.stg_last_error()
    assert smear(h, 0, 1, float("nan"), a, b, None) == -1
    assert smear(h, 0, 1, 0.1, ctypes.c_void_p(8), b, None) == -1
    assert smear(h, 0, 1, 0.1, a, None, None) == -1
    assert smear(h, 2, 1, 0.1, a, b, None) == -1 and b"prec" in L.stg_last_error()
    assert force(h, 0, 2, 0.1, a, b, c, d, 2, None) == -1 and b"kind" in L.stg_last_error()
    assert force(h, 0, 2, 0.1, a, b, c, c, 1, None) == -1 and b"alias" in L.stg_last_error()
    assert force(h, 1, 2, 0.1, a, None, c, d, 1, None) == -1
    assert force(h, 0, 2, -0.51, a, b, c, d, 1, None) == -1
    assert force(h, 4, 2, 0.1, a, b, c, d, 1, None) == -1 and b"prec" in L.stg_last_error()
    L.stg_lattice_destroy(h)


def test_status_strings(L):
    for s in (0, -1, -2, -3, -4, -5, -6, 99):
        assert L.stg_status_string(s)


def test_gauge_and_md_arguments_rejected_before_launch(L):
    rc, h = _lat(L, (4, 4, 4, 4))
    a, b, c = (ctypes.c_void_p(v) for v in (256, 512, 768))
    assert L.stg_gauge_action(None, 5.0, a, ctypes.c_void_p(1024), None) == -1
    assert L.stg_gauge_action(h, 5.0, ctypes.c_void_p(8), ctypes.c_void_p(1024), None) == -1
    assert L.stg_gauge_action(h, float("inf"), a, ctypes.c_void_p(1024), None) == -1
    assert L.stg_gauge_force(h, 0, 5.0, a, a, 0, None) == -1 and b"alias" in L.stg_last_error()
    assert L.stg_gauge_force(h, 1, 5.0, a, b, 3, None) == -1 and b"kind" in L.stg_last_error()
    assert L.stg_gauge_force(h, 3, 5.0, a, b, 0, None) == -1 and b"prec" in L.stg_last_error()
    assert L.stg_md_momenta(h, None, b, None) == -1
    assert L.stg_md_update_links(h, 0.1, a, a, None) == -1 and b"alias" in L.stg_last_error()
    assert L.stg_md_update_links(h, 2.0, a, b, None) == -1 and b"eps" in L.stg_last_error()
    assert L.stg_md_update_momenta(h, 0, float("nan"), a, b, None) == -1
    assert L.stg_md_update_momenta(h, 2, 0.1, a, b, None) == -1
    assert L.stg_complex_convert(10, 0, a, 1, a, None) == -1
    assert L.stg_complex_convert(-1, 0, a, 1, b, None) == -1
    assert L.stg_complex_convert(10, 3, a, 1, b, None) == -1
    assert L.stg_md_kinetic(h, a, None, None) == -1
    assert L.stg_gauge_update(None, a, None, None) == -1
    assert L.stg_dslash(None, 0, a, b, None) == -1
    assert L.stg_dslash(None, 2, a, b, None) == -1 and b"out_parity" in L.stg_last_error()
    assert L.stg_fermion_force_prec(None, 3, 1, None, None, None, 0, None) == -1
    L.stg_lattice_destroy(h)
