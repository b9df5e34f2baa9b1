"""GPU parity of the permutation test (counts of |r_k| >= |r_obs|) against
the FP64 oracle.

Band rule (the reading of the comparison at a finite precision): a pair
whose oracle |r_k| is within 1e-5 of |r_obs| for no k must have the exact
count; otherwise the GPU count lies in [cnt_lo, cnt_hi] with cnt_lo =
#{|r_k| >= |r_obs| + 1e-5} and cnt_hi = #{|r_k| >= |r_obs| - 1e-5}.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
BAND = 1e-5


def _torch():
    import torch
    return torch


def gpu_perm_counts(pcc, X, perms, prec="fp16x3s", ranges=None, Z=None):
    torch = _torch()
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    if Z is None:
        Z = pcc.pcc_standardize(Xd, prec)
    n = X.shape[0]
    P = perms.shape[0]
    dp = torch.from_numpy(np.ascontiguousarray(perms, dtype=np.int32)).cuda()
    cnt = torch.zeros(n * (n - 1) // 2, dtype=torch.int32, device="cuda")
    for a, b in (ranges or [(0, P)]):
        pcc.pcc_perm_test(Z, dp, P, a, b, cnt)
    st = pcc.pcc_sync_status(Z)
    return cnt.cpu().numpy().astype(np.int64), st, Z


def check_band(X, perms, got, I, J):
    c, clo, chi = oracle.perm_counts(X, perms, I, J, delta=BAND)
    n = X.shape[0]
    idx = I * (2 * n - I - 1) // 2 + (J - I - 1)
    g = got[idx]
    exact = clo == chi
    assert np.array_equal(g[exact], c[exact].astype(np.int64)), (
        "exact counts differ", np.nonzero(g[exact] != c[exact])[0][:5])
    assert np.all((g >= clo) & (g <= chi))
    return int(exact.sum()), len(I)


@pytest.mark.parametrize("n,l", [(130, 16), (300, 33), (257, 64),
                                 (520, 200), (400, 256), (300, 300)])
@pytest.mark.parametrize("prec", ["fp16x3s", "bf16x3", "bf16x4"])
def test_perm_counts_parity(pcc_gpu, n, l, prec):
    X = synth.counts_log(n, l, seed=n * 7 + l)
    X[n // 2] = 2.5  # flagged row: counts stay 0
    perms = synth.fisher_yates_perms(40, l, seed=9)
    got, st, _ = gpu_perm_counts(pcc_gpu, X, perms, prec)
    assert st == 0
    I, J = np.triu_indices(n, 1)
    exact, tot = check_band(X, perms, got, I, J)
    assert exact > 0.5 * tot
    flagged = (I == n // 2) | (J == n // 2)
    idx = I * (2 * n - I - 1) // 2 + (J - I - 1)
    assert np.all(got[idx[flagged]] == 0)


def test_identity_permutations_count_all(pcc_gpu):
    X = synth.counts_log(300, 64, seed=3)
    P = 17
    perms = np.tile(np.arange(64, dtype=np.int32), (P, 1))
    got, st, _ = gpu_perm_counts(pcc_gpu, X, perms)
    assert st == 0
    _, flag = oracle.standardize(X)
    I, J = np.triu_indices(300, 1)
    ok = (flag[I] == 0) & (flag[J] == 0)
    assert np.all(got[ok] == P) and np.all(got[~ok] == 0)


@pytest.mark.parametrize("form", [0, 1, 2])
def test_counts_past_16_bits(pcc_gpu, form):
    """70,001 identity permutations: every unflagged pair counts all of
    them, past the 65,535 that one 16-bit register count holds (the forms
    add their register counts to the output at most every 65,534
    permutations of a tile)."""
    X = synth.counts_log(260, 16, seed=5)
    X[7] = 1.0  # flagged row
    P = 70001
    perms = np.tile(np.arange(16, dtype=np.int32), (P, 1))
    before = pcc_gpu.pcc_get_tuning()
    try:
        pcc_gpu.pcc_set_tuning(pair_mma=1, perm_form=form)
        got, st, _ = gpu_perm_counts(pcc_gpu, X, perms)
    finally:
        pcc_gpu.pcc_set_tuning(pair_mma=before["pair_mma"],
                               perm_form=before["perm_form"])
    assert st == 0
    _, flag = oracle.standardize(X)
    I, J = np.triu_indices(260, 1)
    ok = (flag[I] == 0) & (flag[J] == 0)
    assert not ok.all()
    assert np.all(got[ok] == P) and np.all(got[~ok] == 0)


def test_split_ranges_accumulate(pcc_gpu):
    """Counting [0,a) then [a,P) adds up to counting [0,P) (resume)."""
    X = synth.counts_log(400, 128, seed=21)
    perms = synth.fisher_yates_perms(50, 128, seed=22)
    whole, _, _ = gpu_perm_counts(pcc_gpu, X, perms)
    parts, st, _ = gpu_perm_counts(pcc_gpu, X, perms,
                                   ranges=[(0, 13), (13, 31), (31, 50)])
    assert st == 0
    assert np.array_equal(whole, parts)


def test_small_workspace_batches(pcc_gpu, tmp_path):
    """The workspace form with a workspace that holds only 3 permutations
    runs the range as 9 batches; the counts equal the single-batch run
    (fresh process: the budget is read when the library first needs it)."""
    import os
    import subprocess
    import sys
    X = synth.counts_log(260, 96, seed=31)
    perms = synth.fisher_yates_perms(25, 96, seed=32)
    whole, st, _ = gpu_perm_counts(pcc_gpu, X, perms)
    assert st == 0
    np.save(tmp_path / "x.npy", X)
    np.save(tmp_path / "p.npy", perms)
    here = os.path.dirname(os.path.abspath(__file__))
    code = (
        "import sys, numpy as np; sys.path[:0] = [%r, %r]\n"
        "import test_gpu_perm as t, paper_1605_01584_gb300 as pcc\n"
        "pcc.load()\n"
        "got, st, _ = t.gpu_perm_counts(pcc, np.load(%r), np.load(%r))\n"
        "assert st == 0, st\n"
        "np.save(%r, got)\n" % (here, os.path.dirname(here),
                                 str(tmp_path / "x.npy"),
                                 str(tmp_path / "p.npy"),
                                 str(tmp_path / "g.npy")))
    per_k = 260 * 128 * 4
    env = dict(os.environ, PCC_PERM_WS_BYTES=str(3 * per_k),
               PCC_PERM_FORM="1")
    r = subprocess.run([sys.executable, "-c", code], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert np.array_equal(np.load(tmp_path / "g.npy"), whole)


@pytest.mark.parametrize("prec", ["fp16x3s", "bf16x4"])
def test_transposed_form_32_sample_stages(pcc_gpu, tmp_path, prec):
    """The transposed form's variant with six 32-sample B stages
    (PCC_PERM_MN_K=32, read when the library loads: a fresh process) gives
    the workspace form's counts exactly; l = 256 runs 8 stages per pass,
    past the ring's depth, and l = 100 a ragged last stage."""
    import os
    import subprocess
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    for n, l, P in ((400, 256, 17), (300, 100, 6)):
        X = synth.counts_log(n, l, seed=n + l + 71)
        perms = synth.fisher_yates_perms(P, l, seed=l + 72)
        before = pcc_gpu.pcc_get_tuning()
        try:
            pcc_gpu.pcc_set_tuning(pair_mma=1, perm_form=1)
            ref, st, _ = gpu_perm_counts(pcc_gpu, X, perms, prec)
        finally:
            pcc_gpu.pcc_set_tuning(pair_mma=before["pair_mma"],
                                   perm_form=before["perm_form"])
        assert st == 0 and ref.max() > 0
        np.save(tmp_path / "x.npy", X)
        np.save(tmp_path / "p.npy", perms)
        code = (
            "import sys, numpy as np; sys.path[:0] = [%r, %r]\n"
            "import test_gpu_perm as t, paper_1605_01584_gb300 as pcc\n"
            "pcc.load()\n"
            "got, st, _ = t.gpu_perm_counts(pcc, np.load(%r), np.load(%r),"
            " %r)\n"
            "assert st == 0, st\n"
            "np.save(%r, got)\n" % (here, os.path.dirname(here),
                                     str(tmp_path / "x.npy"),
                                     str(tmp_path / "p.npy"), prec,
                                     str(tmp_path / "g.npy")))
        env = dict(os.environ, PCC_PERM_MN_K="32", PCC_PERM_FORM="2",
                   PCC_TC_PAIR="1")
        r = subprocess.run([sys.executable, "-c", code], env=env,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        assert np.array_equal(np.load(tmp_path / "g.npy"), ref), (n, l)


@pytest.mark.parametrize("workspace", [0, 1, 2])
def test_bad_permutation_index_is_reported(pcc_gpu, workspace):
    """Every form checks every index: out of range is read as sample 0 and
    recorded; the other permutations' counts are unaffected."""
    X = synth.counts_log(200, 32, seed=5)
    perms = synth.fisher_yates_perms(4, 32, seed=6)
    good, st0, _ = gpu_perm_counts(pcc_gpu, X, perms[:2])
    perms[2, 7] = 32   # out of range
    perms[3, 0] = -1
    before = pcc_gpu.pcc_get_tuning()
    try:
        pcc_gpu.pcc_set_tuning(perm_form=workspace)
        got, st, _ = gpu_perm_counts(pcc_gpu, X, perms, ranges=[(0, 2)])
        _, st2, _ = gpu_perm_counts(pcc_gpu, X, perms)
    finally:
        pcc_gpu.pcc_set_tuning(perm_form=before["perm_form"])
    assert st0 == 0 and st == 0
    assert np.array_equal(got, good)
    assert st2 == pcc_gpu.PCC_ERR_INVALID_ARG


def test_invalid_ranges(pcc_gpu):
    torch = _torch()
    X = torch.randn((50, 16), device="cuda")
    Z = pcc_gpu.pcc_standardize(X, "fp16x3s")
    dp = torch.zeros((4, 16), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(50 * 49 // 2, dtype=torch.int32, device="cuda")
    for a, b in [(-1, 2), (3, 2), (0, 5)]:
        with pytest.raises(pcc_gpu.PccError):
            pcc_gpu.pcc_perm_test(Z, dp, 4, a, b, cnt)
    Z32 = pcc_gpu.pcc_standardize(X, "fp32")
    with pytest.raises(pcc_gpu.PccError):
        pcc_gpu.pcc_perm_test(Z32, dp, 4, 0, 4, cnt)


def test_perm_full_config_sampled(pcc_gpu):
    """The batched permutation workload: n=4096 x l=256, P=1000 seeded
    Fisher-Yates permutations.  10^5 uniformly sampled pairs plus every pair
    of every planted module against the oracle under the band rule; over
    the whole triangle, 0 <= count <= P (flagged rows are covered by the
    ragged-shape cases: this workload has no constant row)."""
    n, l, P = 4096, 256, 1000
    X, mod = synth.counts_log(n, l, seed=4, return_modules=True)
    perms = synth.fisher_yates_perms(P, l, seed=4)
    got, st, _ = gpu_perm_counts(pcc_gpu, X, perms)
    assert st == 0
    assert got.min() >= 0 and got.max() <= P
    rng = np.random.default_rng(104)
    I = rng.integers(0, n, 100_000)
    J = rng.integers(0, n, 100_000)
    keep = I != J
    I, J = [np.minimum(I, J)[keep]], [np.maximum(I, J)[keep]]
    for m in range(int(mod.max()) + 1):
        g = np.nonzero(mod == m)[0]
        mi, mj = np.triu_indices(len(g), 1)
        I.append(g[mi])
        J.append(g[mj])
    I, J = np.concatenate(I), np.concatenate(J)
    exact, tot = check_band(X, perms, got, I, J)
    assert exact > 0.5 * tot


@pytest.mark.parametrize("n,l,P,prec", [
    (300, 33, 41, "fp16x3s"),    # 3 tile columns: lone diagonal tiles
    (520, 200, 40, "bf16x3"),    # 5 tile columns, resident A
    (400, 300, 17, "bf16x4"),    # rows longer than 256: streamed A
    (129, 64, 7, "fp16x3s"),     # two tile columns, odd P
])
def test_perm_pair_mma_equals_single_cta(pcc_gpu, n, l, P, prec):
    """The CTA-pair form (one 2-SM MMA for two tiles of a tile column, one
    permutation's column rows loaded by each CTA) gives the single-CTA
    form's counts exactly, including the lone last tile of a column, an odd
    number of permutations and a resumed range."""
    pcc = pcc_gpu
    X = synth.counts_log(n, l, seed=n + 5 * l)
    X[n // 3] = 1.5
    perms = synth.fisher_yates_perms(P, l, seed=P)
    before = pcc.pcc_get_tuning()
    try:
        pcc.pcc_set_tuning(pair_mma=0)
        ref, st0, Z = gpu_perm_counts(pcc, X, perms, prec)
        pcc.pcc_set_tuning(pair_mma=1)
        got, st1, _ = gpu_perm_counts(pcc, X, perms, prec, Z=Z)
        part, st2, _ = gpu_perm_counts(pcc, X, perms, prec, Z=Z,
                                       ranges=[(0, 5), (5, P)])
    finally:
        pcc.pcc_set_tuning(pair_mma=before["pair_mma"])
    assert st0 == st1 == st2 == 0
    assert ref.max() > 0
    assert np.array_equal(got, ref)
    assert np.array_equal(part, ref)


@pytest.mark.parametrize("l", [700, 1100])
def test_perm_counts_long_rows(pcc_gpu, l):
    """Rows of 512-1024 samples (the gather keeps four groups of indices
    per lane in registers) and longer (indices read from shared memory),
    both with the streamed A operand."""
    n = 140
    X = synth.counts_log(n, l, seed=l)
    perms = synth.fisher_yates_perms(6, l, seed=l + 1)
    got, st, _ = gpu_perm_counts(pcc_gpu, X, perms, "bf16x3")
    assert st == 0
    I, J = np.triu_indices(n, 1)
    exact, total = check_band(X, perms, got, I, J)
    assert exact > 0.5 * total


@pytest.mark.parametrize("form", [0, 2])
@pytest.mark.parametrize("n,l,P,prec", [
    (300, 33, 41, "fp16x3s"),    # 3 tile columns: a dummy partner tile
    (520, 200, 40, "bf16x3"),    # 5 tile columns
    (129, 64, 7, "fp16x3s"),     # two tile columns, odd P
    (400, 256, 17, "bf16x4"),    # the longest rows of the form, lo.lo
    (260, 96, 1, "fp16x3s"),     # one permutation: a lone pass only
    (700, 130, 2, "bf16x3"),     # one full pass per tile
])
def test_perm_pair_forms_equal_workspace(pcc_gpu, n, l, P, prec, form):
    """CTA pairs that permute the column rows in shared memory (form 0) or
    copy them from a transposed Z (form 2) give the workspace form's counts
    exactly (the same products on the same operands), including a column's
    lone last tile, an odd number of permutations, a single permutation and
    resumed ranges that cut the pass sequence."""
    pcc = pcc_gpu
    X = synth.counts_log(n, l, seed=3 * n + l)
    X[n // 4] = 0.5  # flagged row: counts stay 0
    perms = synth.fisher_yates_perms(P, l, seed=P + l)
    before = pcc.pcc_get_tuning()
    try:
        pcc.pcc_set_tuning(pair_mma=1, perm_form=1)
        ref, st0, Z = gpu_perm_counts(pcc, X, perms, prec)
        pcc.pcc_set_tuning(perm_form=form)
        got, st1, _ = gpu_perm_counts(pcc, X, perms, prec, Z=Z)
        cut = [(0, P // 3), (P // 3, P)] if P > 2 else [(0, 1), (1, P)]
        part, st2, _ = gpu_perm_counts(pcc, X, perms, prec, Z=Z,
                                       ranges=[r for r in cut if r[1] > r[0]])
    finally:
        pcc.pcc_set_tuning(pair_mma=before["pair_mma"],
                           perm_form=before["perm_form"])
    assert st0 == st1 == st2 == 0
    assert ref.max() > 0
    assert np.array_equal(got, ref)
    assert np.array_equal(part, ref)
    I, J = np.triu_indices(n, 1)
    exact, tot = check_band(X, perms, got, I, J)
    assert exact > 0.5 * tot


@pytest.mark.parametrize("form", [0, 2])
@pytest.mark.parametrize("n,l,pair", [(300, 64, 0), (260, 300, 1)])
def test_perm_pair_form_switch_falls_back(pcc_gpu, n, l, pair, form):
    """Where a form without the workspace does not apply (single CTAs, or
    rows longer than 256 samples), selecting it runs the workspace form:
    the counts equal the workspace form's."""
    pcc = pcc_gpu
    X = synth.counts_log(n, l, seed=n + l)
    perms = synth.fisher_yates_perms(9, l, seed=l)
    before = pcc.pcc_get_tuning()
    try:
        pcc.pcc_set_tuning(pair_mma=pair, perm_form=1)
        ref, st0, Z = gpu_perm_counts(pcc, X, perms, "bf16x3")
        pcc.pcc_set_tuning(perm_form=form)
        got, st1, _ = gpu_perm_counts(pcc, X, perms, "bf16x3", Z=Z)
    finally:
        pcc.pcc_set_tuning(pair_mma=before["pair_mma"],
                           perm_form=before["perm_form"])
    assert st0 == st1 == 0
    assert ref.max() > 0
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("form", [1, 2])
def test_perm_graph_replay_follows_restandardize(pcc_gpu, form):
    """A captured permutation test, replayed after Z was standardized again
    from other data outside the graph, counts the new data: the transposed
    form rebuilds its copy of Z inside every captured call."""
    import torch
    pcc = pcc_gpu
    n, l, P = 300, 64, 6
    d1 = torch.from_numpy(synth.counts_log(n, l, seed=11)).cuda()
    d2 = torch.from_numpy(synth.counts_log(n, l, seed=12)).cuda()
    perms = torch.from_numpy(synth.fisher_yates_perms(P, l, seed=13)).cuda()
    cnt = torch.zeros(n * (n - 1) // 2, dtype=torch.int32, device="cuda")
    before = pcc.pcc_get_tuning()
    try:
        pcc.pcc_set_tuning(pair_mma=1, perm_form=form)
        Z = pcc.pcc_standardize(d2, "bf16x3")
        pcc.pcc_perm_test(Z, perms, P, 0, P, cnt)
        want = cnt.cpu().numpy().copy()
        pcc.pcc_standardize(d1, "bf16x3", Z=Z)
        cnt.zero_()
        pcc.pcc_perm_test(Z, perms, P, 0, P, cnt)  # the copy of d1 is built
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                pcc.pcc_perm_test(Z, perms, P, 0, P, cnt, stream=s)
        torch.cuda.synchronize()
        pcc.pcc_standardize(d2, "bf16x3", Z=Z)
        torch.cuda.synchronize()
        cnt.zero_()
        g.replay()
        torch.cuda.synchronize()
        st = pcc.pcc_sync_status(Z)
    finally:
        pcc.pcc_set_tuning(pair_mma=before["pair_mma"],
                           perm_form=before["perm_form"])
    assert st == 0
    assert want.max() > 0
    assert np.array_equal(cnt.cpu().numpy(), want)
