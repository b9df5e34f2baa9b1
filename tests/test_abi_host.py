"""CPU checks of the C-ABI library: it loads, exports every function that
include/pcc.h declares, and its host numbering helpers (the closed forms of
Eq. (14)-(15) and (17)-(19) with integer correction, the code the kernels
also run) agree with the oracle's search-based numbering."""
import ctypes
import os

import numpy as np
import pytest

import oracle
import paper_1605_01584_gb300 as pcc


@pytest.fixture(scope="module")
def lib():
    from paper_1605_01584_gb300 import _build
    _build.build()
    return pcc.load()


def test_exports_every_header_function(lib):
    names = pcc.header_functions()
    assert len(names) >= 16
    raw = ctypes.CDLL(pcc.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert missing == []


def test_status_strings(lib):
    for s in range(7):
        assert pcc.pcc_status_string(s) not in ("", "unknown status")
    assert pcc.pcc_status_string(99) == "unknown status"


def test_pair_numbering_matches_oracle_exhaustive(lib):
    for n in list(range(2, 64)) + [127, 128, 129, 255, 257]:
        assert pcc.pcc_num_pairs(n) == oracle.num_pairs(n)
        for i in range(n):
            for j in range(i + 1, n):
                J = pcc.pcc_pair_index(n, i, j)
                assert J == oracle.pair_index(n, i, j)
                assert pcc.pcc_pair_coords(n, J) == (i, j)
        assert pcc.pcc_pair_index(n, 1, 1) == -1
        assert pcc.pcc_pair_index(n, 0, n) == -1


def test_pair_coords_row_ends_large_n(lib):
    """The last id of every row is where an FP sqrt that rounds low breaks
    Eq. (14); check row starts and ends over whole ranges of rows."""
    for n in (65536, 65537, 100003, 1 << 20, (1 << 24) + 3):
        rows = list(range(0, 2000)) + list(range(n - 2000, n - 1))
        rows += list(np.random.default_rng(n).integers(0, n - 1, 2000))
        for i in rows:
            i = int(i)
            J0 = oracle.pair_index(n, i, i + 1)
            J1 = oracle.pair_index(n, i, n - 1)
            assert pcc.pcc_pair_coords(n, J0) == (i, i + 1)
            assert pcc.pcc_pair_coords(n, J1) == (i, n - 1)


def test_tile_coords_matches_eq9_exhaustive(lib):
    for m in range(1, 90):
        for J in range(m * (m + 1) // 2):
            assert pcc.pcc_tile_coords(m, J) == oracle.job_coords_diag(m, J)
    for m in (512, 513, 4096, 65536):
        for y in list(range(0, 300)) + list(range(m - 300, m)):
            J0 = oracle.job_index_diag(m, y, y)
            J1 = oracle.job_index_diag(m, y, m - 1)
            assert pcc.pcc_tile_coords(m, J0) == (y, y)
            assert pcc.pcc_tile_coords(m, J1) == (y, m - 1)


def test_invalid_numbering_args(lib):
    with pytest.raises(pcc.PccError):
        pcc.pcc_pair_coords(5, 10)
    with pytest.raises(pcc.PccError):
        pcc.pcc_pair_coords(1, 0)
    with pytest.raises(pcc.PccError):
        pcc.pcc_tile_coords(4, 10)
    with pytest.raises(pcc.PccError):
        pcc.pcc_set_wait_limit_ns(0)
    pcc.pcc_set_wait_limit_ns(4_000_000_000)


def test_tuning_knobs_round_trip(lib):
    before = pcc.pcc_get_tuning()
    if "PCC_PERM_FORM" not in os.environ:
        assert before["perm_form"] == pcc.PCC_PERM_TRANSPOSED
    try:
        pcc.pcc_set_tuning(stage_k=64, cluster=1, band_rows=7, cost_c0=11.0,
                           cost_c1=3.0, pair_mma=0, perm_form=0)
        t = pcc.pcc_get_tuning()
        assert t == dict(stage_k=64, cluster=1, band_rows=7, cost_c0=11.0,
                         cost_c1=3.0, pair_mma=0, perm_form=0)
        pcc.pcc_set_tuning()  # zeros keep every value
        assert pcc.pcc_get_tuning() == t
        for bad in (dict(stage_k=48), dict(cluster=3), dict(band_rows=-2),
                    dict(pair_mma=2), dict(perm_form=-1),
                    dict(perm_form=3)):
            with pytest.raises(pcc.PccError):
                pcc.pcc_set_tuning(**bad)
        assert pcc.pcc_get_tuning() == t
    finally:
        pcc.pcc_set_tuning(before["stage_k"], before["cluster"],
                           before["band_rows"], before["cost_c0"],
                           before["cost_c1"], before["pair_mma"],
                           before["perm_form"])
