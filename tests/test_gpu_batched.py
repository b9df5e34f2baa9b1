"""GPU parity of the batched uneven launch (pcc_allpairs_upper_batched):
each matrix against its own single-matrix run and against the oracle, plus
CUDA-graph replay of the launch."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


SHAPES = [(3, 5, "fp16x3s"), (200, 2, "bf16x3"), (513, 33, "fp16x3s"),
          (300, 300, "bf16x3"), (1000, 64, "bf16x1"), (2049, 129, "fp16x3s"),
          (130, 1000, "fp16x3s"), (700, 200, "bf16x4")]


def _setup(pcc, shapes, seed0=900):
    torch = _torch()
    Xs, Zs, Rs = [], [], []
    for b, (n, l, prec) in enumerate(shapes):
        X = synth.counts_log(n, l, seed0 + b)
        if n > 10:
            X[n // 3] = 4.0  # flagged row
        Xd = torch.from_numpy(X).cuda()
        Xs.append(X)
        Zs.append(pcc.pcc_standardize(Xd, prec))
        Rs.append(torch.full((n * (n - 1) // 2,), 7.0, device="cuda"))
    return Xs, Zs, Rs


def test_batched_matches_single_and_oracle(pcc_gpu):
    torch = _torch()
    pcc = pcc_gpu
    Xs, Zs, Rs = _setup(pcc, SHAPES)
    pcc.pcc_allpairs_upper_batched(Zs, Rs)
    assert pcc.pcc_sync_status(Zs[0]) == 0
    for b, (n, l, prec) in enumerate(SHAPES):
        got = Rs[b].cpu().numpy()
        assert not np.any(got == 7.0), b
        single = torch.full_like(Rs[b], 7.0)
        pcc.pcc_allpairs_upper(Zs[b], single)
        single = single.cpu().numpy()
        assert np.array_equal(np.isnan(got), np.isnan(single))
        ok = ~np.isnan(got)
        assert np.array_equal(got[ok], single[ok]), b
        want = oracle.pcc_upper(Xs[b])
        assert np.array_equal(np.isnan(got), np.isnan(want))
        tol = 2e-2 if prec == "bf16x1" else 1e-5
        assert np.max(np.abs(got[ok] - want[ok])) <= tol, (b, prec)


def test_batched_plan_reuse_and_graph_replay(pcc_gpu):
    torch = _torch()
    pcc = pcc_gpu
    Xs, Zs, Rs = _setup(pcc, SHAPES[2:6], seed0=950)
    pcc.pcc_allpairs_upper_batched(Zs, Rs)  # builds the plan
    torch.cuda.synchronize()
    first = [r.clone() for r in Rs]
    for r in Rs:
        r.fill_(7.0)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            pcc.pcc_allpairs_upper_batched(Zs, Rs, stream=s)
    torch.cuda.synchronize()
    for r in Rs:
        r.fill_(7.0)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(first, Rs):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        assert np.array_equal(np.isnan(a), np.isnan(b))
        ok = ~np.isnan(a)
        assert np.array_equal(a[ok], b[ok])
    assert pcc.pcc_sync_status(Zs[0]) == 0


def test_batched_uneven_workload_sampled(pcc_gpu):
    """The first 12 matrices of the 64-matrix uneven workload (n ~
    U{500..20000}, l ~ U{32..2048}), 20,000 sampled pairs each."""
    torch = _torch()
    pcc = pcc_gpu
    shapes = synth.uneven_shapes()[:12]
    Xs, Zs, Rs = [], [], []
    for b, (n, l) in enumerate(shapes):
        X = synth.counts_log(n, l, 5 * 1000 + b)
        Xs.append(X)
        Zs.append(pcc.pcc_standardize(torch.from_numpy(X).cuda(), "auto"))
        Rs.append(torch.empty(n * (n - 1) // 2, device="cuda"))
    pcc.pcc_allpairs_upper_batched(Zs, Rs)
    assert pcc.pcc_sync_status(Zs[0]) == 0
    rng = np.random.default_rng(105)
    worst = 0.0
    for b, (n, l) in enumerate(shapes):
        I = rng.integers(0, n, 20000)
        J = rng.integers(0, n, 20000)
        keep = I != J
        I, J = np.minimum(I, J)[keep], np.maximum(I, J)[keep]
        idx = torch.from_numpy(I * (2 * n - I - 1) // 2 + (J - I - 1)).cuda()
        got = Rs[b][idx].cpu().numpy().astype(np.float64)
        want = oracle.pcc_pairs(Xs[b], I, J)
        assert np.array_equal(np.isnan(got), np.isnan(want))
        ok = ~np.isnan(want)
        worst = max(worst, float(np.max(np.abs(got[ok] - want[ok]))))
    assert worst <= 1e-5, worst


def test_batched_invalid_arguments(pcc_gpu):
    torch = _torch()
    pcc = pcc_gpu
    X = torch.randn((40, 16), device="cuda")
    Z32 = pcc.pcc_standardize(X, "fp32")
    R = torch.empty(40 * 39 // 2, device="cuda")
    with pytest.raises(pcc.PccError):
        pcc.pcc_allpairs_upper_batched([Z32], [R])
    with pytest.raises(pcc.PccError):
        pcc.pcc_allpairs_upper_batched([], [])


def test_batched_pair_mma_equals_single_ctas(pcc_gpu):
    """The pair form (whole tiles to CTA pairs, one 2-SM MMA each) and the
    single-CTA form (units to CTAs) give the same bits; switching the form
    builds a new plan."""
    torch = _torch()
    pcc = pcc_gpu
    Xs, Zs, Rs = _setup(pcc, SHAPES, seed0=950)
    before = pcc.pcc_get_tuning()
    try:
        pcc.pcc_set_tuning(pair_mma=0)
        pcc.pcc_allpairs_upper_batched(Zs, Rs)
        ref = [r.cpu().numpy().copy() for r in Rs]
        for r in Rs:
            r.fill_(7.0)
        pcc.pcc_set_tuning(pair_mma=1)
        pcc.pcc_allpairs_upper_batched(Zs, Rs)
        assert pcc.pcc_sync_status(Zs[0]) == 0
    finally:
        pcc.pcc_set_tuning(pair_mma=before["pair_mma"])
    for b in range(len(SHAPES)):
        got = Rs[b].cpu().numpy()
        assert not np.any(got == 7.0), b
        assert np.array_equal(np.isnan(got), np.isnan(ref[b]))
        ok = ~np.isnan(got)
        assert np.array_equal(got[ok].view(np.uint32),
                              ref[b][ok].view(np.uint32)), b
