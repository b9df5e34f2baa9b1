"""The allocation-free entry point (for callers that may not allocate device
memory, e.g. inside another framework's memory pool) against the regular
standardize + all-pairs path, through the C ABI, on two calls in a row.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the split tensor-core tolerance used by the other GPU tests


def _regular(pcc, Xd, prec):
    import torch
    n = Xd.shape[0]
    Z = pcc.pcc_standardize(Xd, prec)
    R = torch.full((n * (n - 1) // 2,), 7.0, device="cuda")
    pcc.pcc_allpairs_upper(Z, R)
    assert pcc.pcc_sync_status(Z) == 0
    return R.cpu().numpy()


def _compare(got, want):
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.max(np.abs(got[ok].astype(np.float64) -
                         want[ok].astype(np.float64))) <= TOL


@pytest.mark.parametrize("prec", ["fp16x3s", "bf16x3"])
def test_noalloc_matches_regular_path_twice(pcc_gpu, prec):
    import torch
    pcc = pcc_gpu
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    for call, (n, l, seed) in enumerate([(3000, 200, 61), (2049, 333, 62)]):
        X = synth.counts_log(n, l, seed)
        X[n // 5] = 1.5  # a flagged row
        Xd = torch.from_numpy(X).cuda()
        want = _regular(pcc, Xd, prec)
        R = torch.full((n * (n - 1) // 2,), 7.0, device="cuda")
        pcc.pcc_allpairs_upper_noalloc(Xd, R, prec, d_status=st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0, call
        got = R.cpu().numpy()
        assert not np.any(got == 7.0)
        _compare(got, want)


def test_noalloc_rejects_sizes_beyond_the_array(pcc_gpu):
    import torch
    pcc = pcc_gpu
    n, l = 16384, 512  # 4 * n * lpad = 32 MiB alone: over the limit
    Xd = torch.zeros((n, l), device="cuda")
    R = torch.empty(1, device="cuda")
    with pytest.raises(pcc.PccError) as e:
        pcc.pcc_allpairs_upper_noalloc(Xd, R, "fp16x3s")
    assert e.value.status == pcc.PCC_ERR_INVALID_ARG
