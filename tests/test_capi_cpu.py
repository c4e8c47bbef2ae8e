"""The C-ABI library loads and exports every symbol include/pt_ca.h declares (no GPU).

Also checks the host-side argument validation that runs before any CUDA call."""

import os
import re

import pytest

import paper_2501_05520_gb300 as pt
from paper_2501_05520_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:pt_status|const char\*|int)\s+(pt_\w+)\s*\(", txt, re.M)
    return names


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg_build.build()


def test_header_and_binding_agree():
    assert set(_declared()) == set(pt.EXPORTED)


def test_library_exports_every_declared_symbol():
    assert set(pt.exported_symbols()) == set(_declared())


def test_workspace_size_and_capacity_validation():
    n = pt.pt_workspace_size(pt.default_capacity())
    assert n > 0 and n % 256 == 0
    assert pt.pt_workspace_size(pt.default_capacity(max_events=4)) > n
    for bad in (dict(pt.default_capacity(), phi_bins=8),
                dict(pt.default_capacity(), max_ntuplets=1 << 29),
                dict(pt.default_capacity(), max_cells=0),
                dict(pt.default_capacity(), max_hits=1 << 30),
                dict(pt.default_capacity(), reserved=1)):
        with pytest.raises(pt.PtError) as ei:
            pt.pt_workspace_size(bad)
        assert ei.value.status == pt.PT_ERR_INVALID
        assert pt.lib().pt_last_error().decode()


def test_build_is_incremental():
    assert pkg_build.up_to_date()


def test_null_handles_are_rejected_before_any_cuda_call():
    """Every call that takes a context or server answers a NULL handle with
    PT_ERR_INVALID and a message (destroy accepts NULL), without touching CUDA."""
    L = pt.lib()
    calls = {
        "pt_build_doublets": (None, None), "pt_connect_cells": (None, None),
        "pt_find_ntuplets": (None, None), "pt_fit_tracks": (None, None),
        "pt_refit_broken_line": (None, 0.02, 0.02, None),
        "pt_find_vertices": (None, 4, 0.02, None),
        "pt_get_vertices": (None, None, None, None, 0, None, 0),
        "pt_set_modules": (None, None, 0),
        "pt_load_raw": (None, 1, None, None, 0, None),
        "pt_get_hits": (None, None, None, None, None, None, 0, None),
        "pt_get_ntuplets": (None, None, None, None, 0, None, 0),
        "pt_get_tracks": (None, None, 0, None, 0),
        "pt_set_tracing": (None, 1), "pt_get_trace": (None, None, 0, None),
        "pt_submit": (None, 0, None, None, None, None, None),
        "pt_poll": (None, 0, 0, None, None, None, 0, None),
        "pt_server_stats": (None, None, None, None, None),
        "pt_set_layer_pairs": (None, 0, None, None), "pt_set_wait_limit": (None, 1),
        "pt_set_fishbone": (None, 1), "pt_debug_inject": (None, 1),
        "pt_server_counters": (None, None, None, None),
        "pt_router_submit": (None, 0, None, None, None, None, None),
        "pt_router_poll": (None, 0, 0, None, None, None, 0, None),
        "pt_router_stats": (None, None, None, None, None, None),
    }
    for name, args in calls.items():
        assert getattr(L, name)(*args) == pt.PT_ERR_INVALID, name
        assert L.pt_last_error().decode(), name
    assert L.pt_destroy(None) == pt.PT_OK
    assert L.pt_server_destroy(None) == pt.PT_OK
    assert L.pt_router_destroy(None) == pt.PT_OK
