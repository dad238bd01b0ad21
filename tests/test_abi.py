"""C-ABI boundary checks that need no GPU: the library builds, loads, and
exports every entry point that include/lfe.h declares."""
import ctypes
import os
import re

import pytest

from paper_2608_12691_b300 import build as B
from paper_2608_12691_b300 import lfe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lfe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lfe_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ctypes.CDLL(B.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 17
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(lfe.EXPORTED)


def test_binding_structs_match_header():
    # the ctypes mirrors carry every field of the C structs, in order
    src = open(os.path.join(ROOT, "include", "lfe.h")).read()
    body = src[src.index("typedef struct {", src.index("LFE_T_HB")):src.index("} lfe_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"([A-Za-z_0-9]+)(?:\[\d\])?\s*[;,]", body)
    assert [f[0] for f in lfe.Params._fields_] == fields


def test_create_without_gpu_reports_error():
    # on a machine without a GPU the library loads and lfe_create fails cleanly
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2608_12691_b300 import systems as S
    d = S.make_water_box(seed=1, n_waters=20, box_len=1.2, solute=None, n_side=3, r_cut=0.55, grid=16)
    with pytest.raises(lfe.LfeError) as e:
        lfe.System(d)
    assert e.value.code == lfe.LFE_ERR_CUDA
