"""The C-ABI library loads and exports every function include/pt.h declares (no GPU)."""
import ctypes
import os
import re
import shutil

import pytest

from tests.conftest import ROOT


def _declared():
    text = open(os.path.join(ROOT, "include", "pt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pt_[a-z0-9_]+)\s*\(", text)))


def _lib_path():
    from paper_1107_3490_gb300 import build
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        if not os.path.exists(build.LIB):
            pytest.skip("no nvcc and no prebuilt library")
        return build.LIB
    return build.build()


def test_header_declares_the_core_calls():
    names = _declared()
    for core in ("pt_create", "pt_sweep", "pt_energies", "pt_histograms", "pt_destroy", "pt_last_error"):
        assert core in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_lib_path())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1107_3490_gb300 import pt
    assert set(_declared()) <= set(pt._SIGS), set(_declared()) - set(pt._SIGS)


def test_calls_without_gpu_fail_cleanly():
    """On a machine without a GPU, creation reports an error instead of crashing."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except Exception:
        pass
    from paper_1107_3490_gb300 import pt
    _lib_path()
    with pytest.raises(pt.PtError):
        pt.pt_create(10, 2, [0.5, 1.0], 1)
    assert pt.pt_last_error()


def test_library_start_coils_without_gpu():
    """pt_make_coil is host-only: bonds at r0, non-bonded distances >= r0, deterministic."""
    import numpy as np
    from paper_1107_3490_gb300 import pt
    _lib_path()
    a = pt.pt_make_coil(60, 3, 11, 2).astype(np.float64)
    b = pt.pt_make_coil(60, 3, 11, 2).astype(np.float64)
    assert np.array_equal(a, b)
    bonds = np.linalg.norm(a[:, 1:] - a[:, :-1], axis=2)
    assert np.all(np.abs(bonds - 0.7) < 1e-5)
    for r in range(3):
        d = np.linalg.norm(a[r, :, None] - a[r, None, :], axis=2)
        assert d[np.triu_indices(60, 2)].min() >= 0.7 - 1e-5
