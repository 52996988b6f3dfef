"""The C-ABI library loads without a GPU and exports exactly what
include/fishlbm.h declares; the Python binding covers every symbol.  No
compute call is made here."""
import ctypes
import os
import re

from paper_2206_01683_b300 import build, fishlbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fishlbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(fg_[a-z_0-9]+)\s*\(", text))


def test_header_declares_the_five_calls():
    syms = declared_symbols()
    for name in ("fg_create_domain", "fg_set_markers", "fg_step", "fg_get_body_force_torque",
                 "fg_destroy"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    build.build()
    L = ctypes.CDLL(fishlbm.LIB_PATH)
    missing = [s for s in sorted(declared_symbols()) if not hasattr(L, s)]
    assert not missing, missing


def test_binding_signatures_match_header():
    assert set(fishlbm.SIGNATURES) == declared_symbols()
    fishlbm.lib()  # sets restype/argtypes for every symbol


def test_struct_layouts():
    assert ctypes.sizeof(fishlbm.fg_env_desc) == 4 * 3 + 4 + 8 + 4 * 6 + 8 * 3 + 8 + 8 * 3
    assert ctypes.sizeof(fishlbm.fg_frame) == 12 * 8
    assert ctypes.sizeof(fishlbm.fg_options) == 10 * 4


def test_lattice_is_d3q27():
    c, w = fishlbm.fg_lattice()       # host-only call
    assert len({tuple(v) for v in c}) == 27
    assert abs(w.sum() - 1.0) < 1e-15
    assert (c[26 - __import__("numpy").arange(27)] == -c).all()   # opposite of i is 26 - i


def test_ib_iters_out_of_range_is_rejected_before_gpu_work():
    env = fishlbm.env_desc((8, 8, 8), 0.6)
    for m in (0, 9, -1):
        opt = fishlbm.fg_options()
        opt.storage = 0
        opt.ib_iters = m
        opt.eq_order = 2
        opt.use_graphs = 1
        try:
            fishlbm.fg_create_domain([env], opt)
        except fishlbm.FgError as e:
            assert e.status == fishlbm.FG_ERR_INVALID, m
        else:
            raise AssertionError("ib_iters = %d accepted" % m)


def test_invalid_arguments_fail_without_gpu_work():
    bad = fishlbm.env_desc((8, 8, 8), 0.5)      # tau must exceed 1/2
    try:
        fishlbm.fg_create_domain([bad])
    except fishlbm.FgError as e:
        assert e.status == fishlbm.FG_ERR_INVALID
    else:
        raise AssertionError("tau = 0.5 accepted")
    bad = fishlbm.env_desc((8, 8, 2), 0.6, faces=(0, 0, 0, 0, 1, 2))   # open axis of 2 cells
    try:
        fishlbm.fg_create_domain([bad])
    except fishlbm.FgError as e:
        assert e.status == fishlbm.FG_ERR_INVALID
    else:
        raise AssertionError("2-cell open axis accepted")


def test_domain_limits_are_rejected_before_gpu_work():
    """Every documented limit of fg_create_domain fails with FG_ERR_INVALID
    before any GPU work (so these run without a GPU)."""
    ok = fishlbm.env_desc((8, 8, 8), 0.6)
    cases = {
        "no environments": [],
        "4097 environments": [ok] * 4097,
        "zero cells": [fishlbm.env_desc((0, 8, 8), 0.6)],
        "65537 cells on an axis": [fishlbm.env_desc((8, 65537, 1), 0.6)],
        "2^31 slots": [fishlbm.env_desc((2048, 1024, 1024), 0.6)],
        "unknown face": [fishlbm.env_desc((8, 8, 8), 0.6, faces=(0, 0, 0, 0, 4, 4))],
        "unpaired periodic face": [fishlbm.env_desc((8, 8, 8), 0.6, faces=(0, 2, 0, 0, 0, 0))],
        "tau not finite": [fishlbm.env_desc((8, 8, 8), float("nan"))],
        "rho0 <= 0": [fishlbm.env_desc((8, 8, 8), 0.6, rho0=0.0)],
    }
    for name, envs in cases.items():
        try:
            if envs:
                fishlbm.fg_create_domain(envs)
            else:
                out = fishlbm._V()
                fishlbm._check(fishlbm.lib().fg_create_domain(None, 0, None, None, ctypes.byref(out)))
        except fishlbm.FgError as e:
            assert e.status == fishlbm.FG_ERR_INVALID, name
        else:
            raise AssertionError(name + " accepted")


def test_layout_options_are_checked_before_gpu_work():
    """An unknown layout, and the in-place layout with a kernel other than
    the plain one, fail with FG_ERR_INVALID before any GPU work."""
    env = fishlbm.env_desc((8, 8, 8), 0.6)
    bad = [(2, fishlbm.FG_KERNEL_AUTO), (-1, fishlbm.FG_KERNEL_AUTO)]
    bad += [(fishlbm.FG_LAYOUT_AA, v) for v in (fishlbm.FG_KERNEL_STAGED, fishlbm.FG_KERNEL_STAGED512,
                                                 fishlbm.FG_KERNEL_FUSED, fishlbm.FG_KERNEL_OVERLAP)]
    for layout, variant in bad:
        opt = fishlbm.fg_options()
        opt.storage = 0
        opt.layout = layout
        opt.ib_iters = 1
        opt.eq_order = 2
        opt.use_graphs = 1
        opt.kernel_variant = variant
        try:
            fishlbm.fg_create_domain([env], opt)
        except fishlbm.FgError as e:
            assert e.status == fishlbm.FG_ERR_INVALID, (layout, variant)
        else:
            raise AssertionError("layout %d with variant %d accepted" % (layout, variant))


def test_layout_enum_matches_header():
    text = open(os.path.join(ROOT, "include", "fishlbm.h")).read()
    assert "FG_LAYOUT_PULL = 0" in text and "FG_LAYOUT_AA = 1" in text
    assert (fishlbm.FG_LAYOUT_PULL, fishlbm.FG_LAYOUT_AA) == (0, 1)
    assert fishlbm.LAYOUT == {"pull": 0, "aa": 1}
