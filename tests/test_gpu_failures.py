"""Failure detection without a GPU fault: a bounded device wait that runs
out is reported as PCC_ERR_TIMEOUT and the context stays usable; an
allocation that cannot succeed is reported as PCC_ERR_OOM."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cluster,pair,drop", [(2, 1, 1), (1, 0, 1),
                                               (2, 1, 2), (2, 1, 3)])
def test_wait_timeout_is_reported_and_recoverable(pcc_gpu, cluster, pair,
                                                  drop):
    """drop 1: no CTA issues loads; 2 / 3: only the odd / even CTA of each
    pair issues none, so the copies of the other one are in flight (or
    landed) when the waits run out and the end-of-kernel drain must cancel
    the missing share (2) or arm the unarmed one (3) before the CTAs
    leave."""
    import torch
    pcc = pcc_gpu
    X = torch.from_numpy(synth.counts_log(1200, 64, 31)).cuda()
    Z = pcc.pcc_standardize(X, "bf16x3")
    n = 1200
    R = torch.full((n * (n - 1) // 2,), 7.0, device="cuda")
    before = pcc.pcc_get_tuning()
    pcc.pcc_set_tuning(cluster=cluster, pair_mma=pair)
    try:
        pcc.pcc_set_wait_limit_ns(200_000_000)  # 0.2 s
        pcc.pcc_debug_drop_loads(drop)
        pcc.pcc_allpairs_upper(Z, R)
        assert pcc.pcc_sync_status(Z) == pcc.PCC_ERR_TIMEOUT
    finally:
        pcc.pcc_debug_drop_loads(False)
        pcc.pcc_set_wait_limit_ns(4_000_000_000)
        pcc.pcc_set_tuning(cluster=before["cluster"],
                           pair_mma=before["pair_mma"])
    # the status word was cleared by the read and the context still works
    assert pcc.pcc_sync_status(Z) == 0
    pcc.pcc_allpairs_upper(Z, R)
    assert pcc.pcc_sync_status(Z) == 0
    got = R.cpu().numpy()
    ref = torch.full_like(R, 7.0)
    Z32 = pcc.pcc_standardize(X, "fp32")
    pcc.pcc_allpairs_upper(Z32, ref)
    ref = ref.cpu().numpy()
    ok = ~np.isnan(ref)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.max(np.abs(got[ok] - ref[ok])) <= 1e-5


def test_allocation_failure_is_reported(pcc_gpu):
    import torch
    pcc = pcc_gpu
    X = torch.zeros((4, 4), device="cuda")
    # a standardized matrix of 2^31-1 rows x 2^20 samples needs ~8 PB: the
    # allocation fails before anything reads X
    with pytest.raises(pcc.PccError) as e:
        pcc.pcc_standardize(X, "bf16x3", n=(1 << 31) - 1, l=1 << 20,
                            ldx=1 << 20)
    assert e.value.status == pcc.PCC_ERR_OOM
    Z = pcc.pcc_standardize(X + torch.arange(4.0, device="cuda"), "bf16x3")
    assert pcc.pcc_sync_status(Z) == 0


@pytest.mark.parametrize("form", [0, 2])
@pytest.mark.parametrize("drop", [1, 2, 3])
def test_perm_pair_form_wait_timeout_is_reported(pcc_gpu, drop, form):
    """The permutation forms without a workspace under the same hook (0:
    permuted in shared memory, 2: copied from a transposed Z): their A
    producer issues no loads (1), or only the even (2) / odd (3) CTA of
    each pair does; the waits run out, PCC_ERR_TIMEOUT is reported, and
    the next test gives the workspace form's counts."""
    import torch
    pcc = pcc_gpu
    n, l, P = 300, 64, 9
    X = torch.from_numpy(synth.counts_log(n, l, 41)).cuda()
    perms = torch.from_numpy(synth.fisher_yates_perms(P, l, seed=42)).cuda()
    Z = pcc.pcc_standardize(X, "fp16x3s")
    cnt = torch.zeros(n * (n - 1) // 2, dtype=torch.int32, device="cuda")
    before = pcc.pcc_get_tuning()
    try:
        pcc.pcc_set_tuning(pair_mma=1, perm_form=form)
        pcc.pcc_set_wait_limit_ns(200_000_000)  # 0.2 s
        pcc.pcc_debug_drop_loads(drop)
        pcc.pcc_perm_test(Z, perms, P, 0, P, cnt)
        assert pcc.pcc_sync_status(Z) == pcc.PCC_ERR_TIMEOUT
        pcc.pcc_debug_drop_loads(False)
        pcc.pcc_set_wait_limit_ns(4_000_000_000)
        assert pcc.pcc_sync_status(Z) == 0
        cnt.zero_()
        pcc.pcc_perm_test(Z, perms, P, 0, P, cnt)
        assert pcc.pcc_sync_status(Z) == 0
        got = cnt.cpu().numpy()
        pcc.pcc_set_tuning(perm_form=1)
        cnt.zero_()
        pcc.pcc_perm_test(Z, perms, P, 0, P, cnt)
        assert pcc.pcc_sync_status(Z) == 0
    finally:
        pcc.pcc_debug_drop_loads(False)
        pcc.pcc_set_wait_limit_ns(4_000_000_000)
        pcc.pcc_set_tuning(pair_mma=before["pair_mma"],
                           perm_form=before["perm_form"])
    ref = cnt.cpu().numpy()
    assert ref.max() > 0
    assert np.array_equal(got, ref)
