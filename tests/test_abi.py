"""CPU checks of the boundary: the C-ABI library builds for sm_103a, loads, and
exports every entry point that include/fc.h declares (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fc.h")).read()
    return sorted(set(re.findall(r"^FC_API\s+[\w\s\*]+?\b(fc_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2002_07858_gb300 import _build_lib

    path = _build_lib.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("fc_create", "fc_destroy", "fc_load_grid", "fc_set_frac_cov", "fc_run_point", "fc_run_points",
              "fc_submit", "fc_poll", "fc_cancel", "fc_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_2002_07858_gb300 as fc

    assert sorted(fc.binding.EXPORTS) == _declared()
    for n in _declared():
        assert callable(getattr(fc, n))


def test_default_opts_without_gpu(lib):
    import paper_2002_07858_gb300 as fc

    o = fc.fc_default_opts()
    assert (o.max_iter, o.precision, o.top_k, o.fluct, o.cov) == (5, fc.FC_PREC_MIXED, 8, 0, 0)


def test_create_fails_loudly_without_gpu():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2002_07858_gb300 as fc

    with pytest.raises(fc.FCError) as e:
        fc.fc_create(0)
    assert e.value.status == fc.FC_ERR_CUDA


def test_library_is_built_for_sm103a():
    from paper_2002_07858_gb300 import _build_lib

    assert "arch=compute_103a,code=sm_103a" in " ".join(_build_lib.ARCH)
