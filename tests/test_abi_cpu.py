"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, and exports every entry point the public headers declare."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(amp4d_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as G
    path = G._build_module().build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for n in ("amp4d_model_create", "amp4d_set_events", "amp4d_set_norm_points",
              "amp4d_eval_nll", "amp4d_eval_nll_grad"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(lib):
    import paper_2007_14931_gb300 as A
    for n in _declared():
        assert hasattr(A, n), n


def test_create_rejects_bad_arguments_without_gpu(lib):
    """Argument checks run before any CUDA call."""
    import paper_2007_14931_gb300 as A
    h = ctypes.c_void_p()
    rc = A.amp4d_model_create(None, None, 0, 0.6, 2.1, 0, ctypes.byref(h))
    assert rc == A.AMP4D_ERR_ARG
    assert b"null" in A.amp4d_last_error(None)
