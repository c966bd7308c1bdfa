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


def test_binding_records_match_header_layout(tmp_path):
    """The ctypes records of the binding have the C layout of include/amp4d.h
    (sizes and field offsets, as gcc lays the header's structs out)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    import paper_2007_14931_gb300 as A
    recs = {"amp4d_resonance": A.amp4d_resonance, "amp4d_particle_masses": A.amp4d_particle_masses,
            "amp4d_mlp_cfg": A.amp4d_mlp_cfg, "amp4d_hist2d": A.amp4d_hist2d}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "amp4d.h"', "int main(void) {"]
    for name, cls in recs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f[0], name, f[0]))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                 text=True).stdout.splitlines())
    for name, cls in recs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f in cls._fields_:
            assert int(got["%s.%s" % (name, f[0])]) == getattr(cls, f[0]).offset, (name, f[0])


def test_create_rejects_bad_lass_records_without_gpu(lib):
    """The LASS S-wave (Eq. 7-8) applies to a fixed J = 0 K* with a > 0, b >= 0, R >= 0."""
    import dataclasses
    import paper_2007_14931_gb300 as A
    import workloads as W
    bad = [dataclasses.replace(W.LASS, J=1), dataclasses.replace(W.LASS, chain=W.CHAIN_Z, J=1),
           dataclasses.replace(W.LASS, lass_a=0.0), dataclasses.replace(W.LASS, lass_b=-1.0),
           dataclasses.replace(W.LASS, lass_R=float("nan")), dataclasses.replace(W.LASS, shape=7)]
    for r in bad:
        with pytest.raises(A.Amp4dError) as e:
            A.Model([r, W.RESONANCES["K*(892)"]])
        assert e.value.code == A.AMP4D_ERR_ARG
    with pytest.raises(A.Amp4dError) as e:
        A.Model([W.LASS], float_names=["LASS"])
    assert e.value.code == A.AMP4D_ERR_ARG
    assert b"LASS" in A.amp4d_last_error(None)
