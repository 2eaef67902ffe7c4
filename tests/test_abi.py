"""The C-ABI library loads and exports every entry point include/aniso.h
declares; argument validation that needs no GPU behaves as documented."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "aniso.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(aniso3?_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    from paper_1008_0861_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("aniso_create", "aniso_set_field", "aniso_step", "aniso_step_batched"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    for name in _declared():
        assert hasattr(lib, name), name
    import paper_1008_0861_gb300 as P
    assert set(_declared()) == set(P.EXPORTED)


def test_create_validates_arguments(built):
    import paper_1008_0861_gb300 as P
    bad = [dict(nx=2, ny=8), dict(nx=8, ny=2), dict(dx=0.0), dict(dy=-1.0), dict(chi_par=0.0),
           dict(chi_perp=-0.1), dict(chi_perp=2.0), dict(bc=7)]
    for kw in bad:
        args = dict(nx=8, ny=8, dx=1.0, dy=1.0, chi_par=1.0, chi_perp=0.0, bc=1)
        args.update(kw)
        with pytest.raises(P.AnisoError) as ei:
            P.aniso_create(**args)
        assert ei.value.code == P.ANISO_ERR_ARG, kw
    h = P.aniso_create(8, 8, 1.0, 1.0, 1.0)
    try:
        with pytest.raises(P.AnisoError) as ei:
            P.aniso_step(h, 0x1000, 1.0, 1)
        assert ei.value.code == P.ANISO_ERR_STATE
        with pytest.raises(P.AnisoError) as ei:
            P.aniso_set_option(h, P.ANISO_OPT_ORDER, 9)
        assert ei.value.code == P.ANISO_ERR_ARG
        with pytest.raises(P.AnisoError) as ei:
            P.aniso_set_option(h, 99, 0)
        assert ei.value.code == P.ANISO_ERR_ARG
        for a, t in ((-1.0, 1.0), (2.5, 0.0), (float("nan"), 1.0), (2.5, float("inf"))):
            with pytest.raises(P.AnisoError) as ei:
                P.aniso_set_nonlinear(h, a, t)
            assert ei.value.code == P.ANISO_ERR_ARG
        P.aniso_set_nonlinear(h, 2.5, 1.0)
        P.aniso_set_nonlinear(h, 0.0, 1.0)
        P.aniso_set_option(h, P.ANISO_OPT_ORDER, P.ANISO_ORDER_ALTERNATE)
        P.aniso_set_state(h, 5)
        assert P.aniso_get_state(h) == 5
    finally:
        P.aniso_destroy(h)


def test_create3_validates_arguments(built):
    import paper_1008_0861_gb300 as P
    bad = [dict(nx=2), dict(ny=2), dict(nz=2), dict(dx=0.0), dict(dz=-1.0), dict(chi_par=0.0),
           dict(chi_perp=2.0), dict(bc=P.ANISO_BC_DIRICHLET)]
    for kw in bad:
        args = dict(nx=8, ny=8, nz=8, dx=1.0, dy=1.0, dz=1.0, chi_par=1.0, chi_perp=0.0, bc=1)
        args.update(kw)
        with pytest.raises(P.AnisoError) as ei:
            P.aniso3_create(**args)
        assert ei.value.code == P.ANISO_ERR_ARG, kw
    h = P.aniso3_create(8, 12, 10, 1.0, 1.0, 1.0, 1.0)
    try:
        with pytest.raises(P.AnisoError) as ei:
            P.aniso3_step(h, 0x1000, 1.0, 1)
        assert ei.value.code == P.ANISO_ERR_STATE
        with pytest.raises(P.AnisoError) as ei:
            P.aniso3_set_option(h, P.ANISO_OPT_SCHEME, P.ANISO_SCHEME_EXPLICIT)
        assert ei.value.code == P.ANISO_ERR_UNSUPPORTED
        with pytest.raises(P.AnisoError) as ei:
            P.aniso3_set_option(h, P.ANISO_OPT_KAHAN, 1)
        assert ei.value.code == P.ANISO_ERR_UNSUPPORTED
        with pytest.raises(P.AnisoError) as ei:
            P.aniso3_set_option(h, 99, 0)
        assert ei.value.code == P.ANISO_ERR_ARG
        P.aniso3_set_option(h, P.ANISO_OPT_SCHEME, P.ANISO_SCHEME_4STEP)
        P.aniso3_set_option(h, P.ANISO_OPT_PRECISION, P.ANISO_PREC_FP32)
        # nz = 10 is not a multiple of the 4-cell FP32 vector: refused before any allocation
        with pytest.raises(P.AnisoError) as ei:
            P.aniso3_set_field(h, 0x1000, 0x1000, 0x1000)
        assert ei.value.code == P.ANISO_ERR_UNSUPPORTED and "nz=10" in str(ei.value)
    finally:
        P.aniso3_destroy(h)


def test_requests_beyond_the_limits_are_refused_before_any_allocation(built):
    import paper_1008_0861_gb300 as P
    with pytest.raises(P.AnisoError) as ei:
        P.aniso_batch_create([])
    assert ei.value.code == P.ANISO_ERR_ARG
    # a row longer than the on-chip line limit (16384 cells in FP32)
    h = P.aniso_create(16388, 8, 1.0, 1.0, 1.0)
    try:
        P.aniso_set_option(h, P.ANISO_OPT_PRECISION, P.ANISO_PREC_FP32)
        with pytest.raises(P.AnisoError) as ei:
            P.aniso_set_field(h, 0x1000, 0x1000)
        assert ei.value.code == P.ANISO_ERR_UNSUPPORTED
    finally:
        P.aniso_destroy(h)
    # a 3-D line longer than the 3-D kernel takes (2048 cells in FP32)
    h3 = P.aniso3_create(2052, 8, 8, 1.0, 1.0, 1.0, 1.0)
    try:
        P.aniso3_set_option(h3, P.ANISO_OPT_PRECISION, P.ANISO_PREC_FP32)
        with pytest.raises(P.AnisoError) as ei:
            P.aniso3_set_field(h3, 0x1000, 0x1000, 0x1000)
        assert ei.value.code == P.ANISO_ERR_UNSUPPORTED
    finally:
        P.aniso3_destroy(h3)


def test_library_does_not_reference_the_oracle(built):
    data = open(built, "rb").read()
    assert b"or_xsweep" not in data and b"liboracle" not in data


def test_autotune_candidate_table(built):
    """The tuner's candidates are valid option values (no GPU needed)."""
    import paper_1008_0861_gb300 as P
    k = 0
    while True:
        try:
            fast, warps, seg = P.aniso_autotune_candidate(k)
        except P.AnisoError as e:
            assert e.code == P.ANISO_ERR_ARG
            break
        assert fast in (1, 3) and warps in (0, 1, 2, 4, 8) and 1 <= seg <= 64
        k += 1
    assert k >= 4
