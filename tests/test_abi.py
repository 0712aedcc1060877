"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point that include/qsw.h declares, and its host helpers (theta
table, Code Fragment 3.1) agree with the oracle."""
import os
import re

import numpy as np
import pytest

from tests.libbuild import ensure_built

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    ensure_built()
    from paper_2003_02450_gb300 import qsw
    return qsw


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "qsw.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qsw_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(capi):
    lib = capi.lib()
    names = declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(capi._SIGNATURES)


@pytest.mark.parametrize("precision", ["c128", "c64"])
def test_theta_table_matches_oracle(capi, precision):
    from oracle import expmv
    got = capi.qsw_theta_table(precision)
    name = "double" if precision == "c128" else "single"
    ref = np.array([expmv.THETA[name][m] for m in range(1, 56)])
    assert np.max(np.abs(got - ref) / ref) <= 1e-13


NORM_CASES = [
    [4.0, 10.0, 20.0, 40.0, 90.0, 200.0, 400.0, 900.0, 1800.0],      # cycle-like
    [64.9, 1500.0, 4.0e4, 9.0e5, 2.0e7, 4.0e8, 9.0e9, 2.0e11, 4.0e12],
    [8.0, 50.0, 300.0, 2000.0, 1.2e4, 7.0e4, 4.0e5, 2.5e6, 1.5e7],
    [1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0],
    [0.0] * 9,
]


@pytest.mark.parametrize("norms", NORM_CASES)
@pytest.mark.parametrize("t", [0.0, 0.05, 1.0, 5.0, 37.5, 500.0])
@pytest.mark.parametrize("n0", [1, 4])
def test_select_params_matches_oracle(capi, norms, t, n0):
    from oracle import expmv
    import scipy.sparse as sp
    info = expmv.NormInfo(sp.csr_matrix((2, 2)), norms=norms)
    for prec, name in (("c128", "double"), ("c64", "single")):
        assert capi.qsw_select_params(norms, t, n0, prec) == expmv.select_params(info, t, n0, name)


def test_select_params_rejects_bad_input(capi):
    with pytest.raises(capi.QswError) as ei:
        capi.qsw_select_params([1.0] * 9, -1.0)
    assert ei.value.name == "QSW_ERR_INVALID_ARG"
    with pytest.raises(capi.QswError):
        capi.qsw_theta_table(7)


def test_create_fails_cleanly_without_gpu(capi):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(capi.QswError):
        capi.qsw_create(0)
