"""The allocation-free entry point, for callers that may not allocate device
memory (code inside another framework's memory pool, programs whose device
budget is fixed at start-up, paths that cannot take cudaMalloc's implicit
synchronisation), through the C ABI, on two calls in a row.

It runs the same standardize and pair kernels as pcc_standardize +
pcc_allpairs_upper on the same layout, so its output must equal theirs bit
for bit (NaN positions included), and both must match the FP64 oracle
within the split form's 1e-5.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the split tensor-core tolerance used by the other GPU tests
SENT = 7.0


def _regular(pcc, Xd, prec):
    import torch
    n = Xd.shape[0]
    Z = pcc.pcc_standardize(Xd, prec)
    R = torch.full((n * (n - 1) // 2,), SENT, device="cuda")
    pcc.pcc_allpairs_upper(Z, R)
    assert pcc.pcc_sync_status(Z) == 0
    return R.cpu().numpy()


def _same_bits(got, want):
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.array_equal(got[ok].view(np.uint32), want[ok].view(np.uint32))


def _vs_oracle(got, X, tol):
    want = oracle.pcc_upper(X)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.max(np.abs(got[ok].astype(np.float64) - want[ok])) <= tol


def _input(n, l, seed, pad):
    """n x l FP32 counts with a flagged row; pad > 0 leaves a gap of pad
    columns after each row (leading dimension l + pad)."""
    X = synth.counts_log(n, l, seed)
    X[n // 5] = 1.5  # a flagged row
    if pad:
        W = np.full((n, l + pad), np.float32(-3e8), dtype=np.float32)
        W[:, :l] = X
        return X, W
    return X, X


@pytest.mark.parametrize("prec,pad,with_status", [
    ("fp16x3s", 0, True), ("bf16x3", 0, True), ("bf16x4", 0, True),
    ("bf16x1", 0, True), ("fp16x3s", 5, True), ("bf16x3", 0, False),
])
def test_noalloc_matches_regular_path_twice(pcc_gpu, prec, pad,
                                            with_status):
    import torch
    pcc = pcc_gpu
    st = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    for call, (n, l, seed) in enumerate([(3000, 200, 61), (2049, 333, 62)]):
        X, W = _input(n, l, seed, pad)
        Wd = torch.from_numpy(W).cuda()
        Xd = Wd[:, :l]  # a view: leading dimension l + pad
        want = _regular(pcc, Xd, prec)
        R = torch.full((n * (n - 1) // 2,), SENT, device="cuda")
        pcc.pcc_allpairs_upper_noalloc(Xd, R, prec,
                                       d_status=st if with_status else None)
        torch.cuda.synchronize()
        if with_status:
            assert int(st.item()) == 0, call  # set to 0 by the call
        got = R.cpu().numpy()
        assert not np.any(got == SENT)
        _same_bits(got, want)
        if prec != "bf16x1":  # single BF16 is reported, not accepted
            _vs_oracle(got, X, TOL)


def test_noalloc_reports_a_wait_timeout(pcc_gpu):
    """A device wait that runs out is reported through d_status (the test
    hook makes the pair kernel's producer issue no loads, so the first
    operand wait of every CTA runs out; nothing faults or hangs), and the
    next call works."""
    import torch
    pcc = pcc_gpu
    n, l = 1500, 96
    X, _ = _input(n, l, 63, 0)
    Xd = torch.from_numpy(X).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    R = torch.full((n * (n - 1) // 2,), SENT, device="cuda")
    try:
        pcc.pcc_set_wait_limit_ns(200_000_000)  # 0.2 s
        pcc.pcc_debug_drop_loads(True)
        pcc.pcc_allpairs_upper_noalloc(Xd, R, "fp16x3s", d_status=st)
        torch.cuda.synchronize()
        assert int(st.item()) == pcc.PCC_ERR_TIMEOUT
    finally:
        pcc.pcc_debug_drop_loads(False)
        pcc.pcc_set_wait_limit_ns(4_000_000_000)
    pcc.pcc_allpairs_upper_noalloc(Xd, R, "fp16x3s", d_status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    _same_bits(R.cpu().numpy(), _regular(pcc, Xd, "fp16x3s"))


def test_noalloc_rejects_sizes_beyond_the_array(pcc_gpu):
    import torch
    pcc = pcc_gpu
    n, l = 16384, 512  # 4 * n * lpad = 32 MiB alone: over the limit
    Xd = torch.zeros((n, l), device="cuda")
    R = torch.empty(1, device="cuda")
    with pytest.raises(pcc.PccError) as e:
        pcc.pcc_allpairs_upper_noalloc(Xd, R, "fp16x3s")
    assert e.value.status == pcc.PCC_ERR_INVALID_ARG
