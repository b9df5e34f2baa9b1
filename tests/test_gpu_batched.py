"""GPU parity of the batched uneven launch (pcc_allpairs_upper_batched):
each matrix against its own single-matrix run and against the oracle, plus
CUDA-graph replay of the launch."""
import json

import numpy as np
import pytest

import oracle
import synth
from gpu_compare import max_abs_diff

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


# (300, 1100) and (260, 2100): rows past 1,024 samples, two accumulators
SHAPES = [(3, 5, "fp16x3s"), (200, 2, "bf16x3"), (513, 33, "fp16x3s"),
          (300, 300, "bf16x3"), (1000, 64, "bf16x1"), (2049, 129, "fp16x3s"),
          (130, 1000, "fp16x3s"), (700, 200, "bf16x4"), (300, 1100, "fp16x3s"),
          (260, 2100, "bf16x3")]


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
    """The whole 64-matrix uneven workload (n ~ U{500..20000}, l ~
    U{32..2048}) in the launches the benchmark times: one batched
    standardize, one batched pair launch.  Per matrix, 10^5 uniformly
    sampled pairs plus every pair of its first 5 planted modules (where
    |r| -> 1 and the split error peaks) against the oracle."""
    torch = _torch()
    pcc = pcc_gpu
    shapes = synth.uneven_shapes()
    gen = synth.counts_log_many(shapes, [5 * 1000 + b
                                         for b in range(len(shapes))],
                                return_modules=True)
    Xs = [torch.from_numpy(X).cuda() for X, _ in gen]
    Zs = pcc.pcc_standardize_batched(Xs, "auto")
    Rs = [torch.empty(n * (n - 1) // 2, device="cuda") for n, _ in shapes]
    pcc.pcc_allpairs_upper_batched(Zs, Rs)
    assert pcc.pcc_sync_status(Zs[0]) == 0
    rng = np.random.default_rng(105)
    worst, checked = 0.0, 0
    for b, ((n, l), (X, mod)) in enumerate(zip(shapes, gen)):
        I = rng.integers(0, n, 100_000)
        J = rng.integers(0, n, 100_000)
        keep = I != J
        I, J = [np.minimum(I, J)[keep]], [np.maximum(I, J)[keep]]
        for m in range(min(int(mod.max()) + 1, 5)):
            g = np.nonzero(mod == m)[0]
            u, v = np.triu_indices(len(g), 1)
            I.append(g[u])
            J.append(g[v])
        I, J = np.concatenate(I), np.concatenate(J)
        idx = torch.from_numpy(I * (2 * n - I - 1) // 2 + (J - I - 1)).cuda()
        got = Rs[b][idx].cpu().numpy().astype(np.float64)
        want = oracle.pcc_pairs(X, I, J)
        assert np.array_equal(np.isnan(got), np.isnan(want)), b
        ok = ~np.isnan(want)
        err = float(np.max(np.abs(got[ok] - want[ok])))
        assert err <= 1e-5, (b, n, l, err)
        worst = max(worst, err)
        checked += int(ok.sum())
    # every pair of every matrix against its FP64 CUDA-core triangle
    worst_all = 0.0
    for b, (n, l) in enumerate(shapes):
        Z64 = pcc.pcc_standardize(Xs[b], "fp64")
        R64 = torch.empty(n * (n - 1) // 2, dtype=torch.float64,
                          device="cuda")
        pcc.pcc_allpairs_upper(Z64, R64)
        assert pcc.pcc_sync_status(Z64) == 0
        e, nan_differs = max_abs_diff(Rs[b], R64)
        assert not nan_differs, b
        assert e <= 1e-5, (b, n, l, e)
        worst_all = max(worst_all, e)
        Z64.close()
        del R64
    print(json.dumps({"batched_workload_max_abs_dr": worst,
                      "pairs_checked": checked,
                      "all_pairs_max_abs_dr_vs_fp64_path": worst_all}))


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


def _zbytes(pcc, Z):
    """The stored halves (or z) and flags of Z as raw bytes on the host."""
    import ctypes
    torch = _torch()
    info, buf = Z.info(), Z.buffers()
    n, lpad = info["n"], info["lpad"]
    libcuda = ctypes.CDLL("libcuda.so.1")
    out = {}
    for key, per in (("hi", 2), ("lo", 2), ("z", 4 if info["prec"] == 1
                                            else 8), ("flags", 0)):
        if not buf[key]:
            continue
        nb = n if key == "flags" else n * lpad * per
        t = torch.empty(nb, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        assert libcuda.cuMemcpy(ctypes.c_uint64(t.data_ptr()),
                                ctypes.c_uint64(buf[key]),
                                ctypes.c_size_t(nb)) == 0
        out[key] = t.cpu().numpy()
    return out


def test_standardize_batched_equals_single_calls(pcc_gpu):
    """One launch per stored form over many matrices (uneven n and l, an
    odd row pitch, AUTO resolving to FP16X3S at every l) gives the
    bits of one pcc_standardize per matrix, reuses matching Zmats and
    replaces one whose shape changed."""
    torch = _torch()
    pcc = pcc_gpu
    shapes = [(500, 40), (3, 5), (2049, 129), (700, 2100), (130, 1000),
              (1000, 513), (64, 64), (4000, 300)]
    Xs = []
    for b, (n, l) in enumerate(shapes):
        X = synth.counts_log(n, l, 700 + b)
        X[n // 2] = 3.0  # flagged row
        if b == 5:  # odd pitch: rows not 16-byte aligned
            wide = np.zeros((n, l + 1), dtype=np.float32)
            wide[:, :l] = X
            Xs.append(torch.from_numpy(wide).cuda()[:, :l])
        else:
            Xs.append(torch.from_numpy(X).cuda())
    for prec in ("auto", "bf16x3", "bf16x1", "fp32", "fp64"):
        Zb = pcc.pcc_standardize_batched(Xs, prec)
        for b, X in enumerate(Xs):
            Zs = pcc.pcc_standardize(X, prec)
            assert Zb[b].info() == Zs.info(), (prec, b)
            got, want = _zbytes(pcc, Zb[b]), _zbytes(pcc, Zs)
            assert got.keys() == want.keys()
            for k in want:
                assert np.array_equal(got[k], want[k]), (prec, b, k)
            Zs.close()
        # a second call reuses every matching Zmat in place
        again = pcc.pcc_standardize_batched(Xs, prec, Zs=Zb)
        assert all(a is z for a, z in zip(again, Zb))
    Zb = pcc.pcc_standardize_batched(Xs, "auto")
    auto = {b: Zb[b].info()["prec"] for b in range(len(shapes))}
    # FP16X3S at every l (long rows accumulate in chunks)
    assert set(auto.values()) == {pcc.PCC_PREC_FP16X3S}
    X2 = list(Xs)
    X2[0] = torch.from_numpy(synth.counts_log(600, 40, 9)).cuda()
    Zc = pcc.pcc_standardize_batched(X2, "auto", Zs=Zb)
    assert Zc[0] is not Zb[0] and Zc[0].info()["n"] == 600
    assert all(Zc[b] is Zb[b] for b in range(1, len(shapes)))


def test_standardize_batched_invalid_arguments(pcc_gpu):
    torch = _torch()
    pcc = pcc_gpu
    good = torch.rand((10, 8), device="cuda")
    bad = torch.rand((1, 8), device="cuda")  # n < 2
    with pytest.raises(pcc.PccError):
        pcc.pcc_standardize_batched([good, bad])
    with pytest.raises(pcc.PccError):
        pcc.pcc_standardize_batched([])


TUNED = [(1100, 300, "fp16x3s"), (700, 1100, "fp16x3s"), (2049, 96, "bf16x3"),
         (520, 64, "fp16x3s")]
CHOICES = [(1, 2), (0, 5), (0, 1), (1, 32)]  # (pair, band rows) per matrix


def _single(pcc, Z, R, pair, band):
    """pcc_allpairs_upper of one matrix under the given form and band."""
    torch = _torch()
    old = pcc.pcc_get_tuning()
    try:
        pcc.pcc_set_tuning(cluster=2 if pair else 1, band_rows=band,
                           pair_mma=pair)
        out = torch.full_like(R, 7.0)
        pcc.pcc_allpairs_upper(Z, out)
        assert pcc.pcc_sync_status(Z) == 0
    finally:
        pcc.pcc_set_tuning(old["stage_k"], old["cluster"], old["band_rows"],
                           pair_mma=old["pair_mma"])
    return out.cpu().numpy()


def test_batched_per_matrix_choices(pcc_gpu):
    """Matrices of one batch under different tuned shapes (CTA pairs or
    single CTAs, band rows 1 to 32): two persistent launches, each matrix
    bit-equal to its single run under the same choice and within 1e-5 of
    the oracle; graph replay of the tuned call gives the same bits."""
    torch = _torch()
    pcc = pcc_gpu
    Xs, Zs, Rs = _setup(pcc, TUNED, seed0=950)
    used = pcc.pcc_allpairs_upper_batched(Zs, Rs, choices=CHOICES)
    assert used == CHOICES
    assert pcc.pcc_sync_status(Zs[0]) == 0
    first = [R.cpu().numpy() for R in Rs]
    for b, (n, l, prec) in enumerate(TUNED):
        got = first[b]
        assert not np.any(got == 7.0), b
        single = _single(pcc, Zs[b], Rs[b], *CHOICES[b])
        assert np.array_equal(np.isnan(got), np.isnan(single))
        ok = ~np.isnan(got)
        assert np.array_equal(got[ok].view(np.uint32),
                              single[ok].view(np.uint32)), b
        want = oracle.pcc_upper(Xs[b])
        assert np.array_equal(np.isnan(got), np.isnan(want))
        assert np.max(np.abs(got[ok] - want[ok])) <= 1e-5, b
    for R in Rs:
        R.fill_(7.0)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pcc.pcc_allpairs_upper_batched(Zs, Rs, choices=CHOICES)
    g.replay()
    torch.cuda.synchronize()
    for b in range(len(TUNED)):
        got = Rs[b].cpu().numpy()
        ok = ~np.isnan(got)
        assert np.array_equal(got[ok].view(np.uint32),
                              first[b][ok].view(np.uint32)), b


def test_batched_default_consults_the_tune_cache(pcc_gpu):
    """With a tune cache holding entries for some shapes, the default call
    gives those matrices the cached best choice at the batched kernel's
    stage size and the rest the current knobs."""
    pcc = pcc_gpu
    from paper_1605_01584_gb300 import autotune
    Xs, Zs, Rs = _setup(pcc, TUNED, seed0=960)
    t = pcc.pcc_get_tuning()
    sk, other = t["stage_k"], 96 - t["stage_k"]  # 32 <-> 64
    cache = {}
    for (n, l, prec), (pair, band) in zip(TUNED[:2], [(0, 4), (1, 16)]):
        cache[autotune.bucket(n, l, prec)] = {
            "best": {"stage_k": other, "cluster": 1, "band_rows": 8,
                     "pair_mma": 0, "ms": 0.5},
            "all": [{"stage_k": other, "cluster": 1, "pair_mma": 0,
                     "band_rows": 8, "ms": 0.5},
                    {"stage_k": sk, "cluster": 2 if pair else 1,
                     "pair_mma": pair, "band_rows": band, "ms": 0.6},
                    {"stage_k": sk, "cluster": 1, "pair_mma": 0,
                     "band_rows": 64, "ms": 0.9}]}
    default = (1 if t["pair_mma"] and t["cluster"] == 2 else 0,
               t["band_rows"])
    used = pcc.pcc_allpairs_upper_batched(Zs, Rs, cache=cache)
    assert used == [(0, 4), (1, 16), default, default]
    assert pcc.pcc_sync_status(Zs[0]) == 0
    for b in range(len(TUNED)):
        got = Rs[b].cpu().numpy()
        single = _single(pcc, Zs[b], Rs[b], *used[b])
        ok = ~np.isnan(got)
        assert np.array_equal(got[ok].view(np.uint32),
                              single[ok].view(np.uint32)), b


def test_batched_rejects_bad_choices(pcc_gpu):
    pcc = pcc_gpu
    _, Zs, Rs = _setup(pcc, TUNED[:2], seed0=970)
    for bad in ([(2, 8), (1, 8)], [(1, 0), (1, 8)], [(1, 5000), (0, 8)]):
        with pytest.raises(pcc.PccError) as e:
            pcc.pcc_allpairs_upper_batched(Zs, Rs, choices=bad)
        assert e.value.status == pcc.PCC_ERR_INVALID_ARG
