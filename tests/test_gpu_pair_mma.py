"""The CTA-pair form of the tensor-core pair kernel gives the same results
as independent CTAs.

A super-tile's two 128-row halves either run on two independent CTAs (one
M = 128 MMA each, every CTA loading all 256 column rows) or on a CTA pair
as one 2-SM MMA (tcgen05.mma.cta_group::2, M = 256; each CTA loads only its
half of the column rows).  Each accumulator sees the same products in the
same K order and the epilogue is shared, so the outputs must agree bit for
bit: over every split form, ragged shapes, tile ranges, chunked
accumulation of long rows, the fused edge list and the two-matrix form.
One case is also held against the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SENT = 7.0


def _data(n, l, seed):
    X = synth.counts_log(n, l, seed, dtype=np.float32)
    X[n // 3] = 2.5  # a flagged (constant) row
    return X


class _Form:
    """K = 32 stages; CTA pairs with the 2-SM MMA (pair = 1) or independent
    CTAs (pair = 0); restores the knobs."""

    def __init__(self, pcc, pair, band=0):
        self.pcc, self.pair, self.band = pcc, pair, band

    def __enter__(self):
        self.old = self.pcc.pcc_get_tuning()
        self.pcc.pcc_set_tuning(stage_k=32, cluster=2 if self.pair else 1,
                                band_rows=self.band, pair_mma=self.pair)

    def __exit__(self, *a):
        o = self.old
        self.pcc.pcc_set_tuning(o["stage_k"], o["cluster"], o["band_rows"],
                                pair_mma=o["pair_mma"])


def _upper(pcc, Z, n, ranges=None):
    import torch
    R = torch.full((n * (n - 1) // 2,), SENT, device="cuda")
    if ranges is None:
        pcc.pcc_allpairs_upper(Z, R)
    else:
        for a, b in ranges:
            pcc.pcc_allpairs_upper(Z, R, a, b)
    st = pcc.pcc_sync_status(Z)
    assert st == 0, pcc.pcc_status_string(st)
    return R.cpu().numpy()


def _same_bits(a, b, what):
    assert np.array_equal(np.isnan(a), np.isnan(b)), what
    ok = ~np.isnan(a)
    assert np.array_equal(a[ok].view(np.uint32), b[ok].view(np.uint32)), what


@pytest.mark.parametrize("prec", ["fp16x3s", "bf16x3", "bf16x4", "bf16x1"])
@pytest.mark.parametrize("n,l", [(300, 40), (1000, 130), (2300, 96)])
def test_pair_mma_equals_single_cta_bits(pcc_gpu, prec, n, l):
    import torch
    pcc = pcc_gpu
    X = torch.from_numpy(_data(n, l, 80 + n + l)).cuda()
    Z = pcc.pcc_standardize(X, prec)
    with _Form(pcc, 0, band=3):
        ref = _upper(pcc, Z, n)
    with _Form(pcc, 1, band=3):
        got = _upper(pcc, Z, n)
    assert not np.any(got == SENT)
    _same_bits(got, ref, f"{prec} {n}x{l}")


def test_pair_mma_tile_ranges(pcc_gpu):
    import torch
    pcc = pcc_gpu
    n, l = 1900, 64
    X = torch.from_numpy(_data(n, l, 81)).cuda()
    Z = pcc.pcc_standardize(X, "fp16x3s")
    T = Z.num_tiles()
    with _Form(pcc, 0, band=2):
        ref = _upper(pcc, Z, n)
    cuts = [0, 1, 3, 4, 9, 16, T - 2, T]
    with _Form(pcc, 1, band=2):
        got = _upper(pcc, Z, n, list(zip(cuts, cuts[1:])))
        part = _upper(pcc, Z, n, [(4, 9)])
    _same_bits(got, ref, "union of ranges")
    w = part != SENT
    assert np.any(w) and not np.all(w)
    _same_bits(part[w], ref[w], "one range")


def test_pair_mma_two_accumulators_and_oracle(pcc_gpu):
    """l > 1024: each unit accumulates in two chunks, folded by the
    epilogue."""
    import torch
    pcc = pcc_gpu
    n, l = 700, 1100
    Xh = _data(n, l, 82)
    X = torch.from_numpy(Xh).cuda()
    Z = pcc.pcc_standardize(X, "bf16x3")
    with _Form(pcc, 0):
        ref = _upper(pcc, Z, n)
    with _Form(pcc, 1):
        got = _upper(pcc, Z, n)
    _same_bits(got, ref, "two accumulators")
    want = oracle.pcc_upper(Xh)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.max(np.abs(got[ok] - want[ok])) <= 1e-5


def test_pair_mma_edges(pcc_gpu):
    import torch
    pcc = pcc_gpu
    n, l = 2100, 80
    X = torch.from_numpy(_data(n, l, 83)).cuda()
    Z = pcc.pcc_standardize(X, "fp16x3s")
    cap = 1 << 18

    def run():
        E = torch.zeros(cap * pcc.EDGE_BYTES, dtype=torch.uint8,
                        device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        R = torch.full((n * (n - 1) // 2,), SENT, device="cuda")
        pcc.pcc_threshold_edges(Z, 0.6, E, cap, cnt, R)
        assert pcc.pcc_sync_status(Z) == 0
        c = int(cnt.item())
        i, j, r = pcc.edges_view(E, c)
        return c, sorted(zip(i.tolist(), j.tolist(), r.tolist())), \
            R.cpu().numpy()

    with _Form(pcc, 0):
        c0, e0, r0 = run()
    with _Form(pcc, 1):
        c1, e1, r1 = run()
    assert c0 > 0 and c1 == c0 and e1 == e0
    _same_bits(r1, r0, "R with edges")


def test_pair_mma_cross(pcc_gpu):
    import torch
    pcc = pcc_gpu
    X = torch.from_numpy(_data(1500, 72, 84)).cuda()
    Y = torch.from_numpy(_data(1100, 72, 85)).cuda()
    ZX = pcc.pcc_standardize(X, "fp16x3s")
    ZY = pcc.pcc_standardize(Y, "fp16x3s")

    def run():
        R = torch.full((1500, 1100), SENT, device="cuda")
        pcc.pcc_cross_allpairs(ZX, ZY, R)
        assert pcc.pcc_sync_status(ZX) == 0
        return R.cpu().numpy().ravel()

    with _Form(pcc, 0, band=2):
        ref = run()
    with _Form(pcc, 1, band=2):
        got = run()
    assert not np.any(got == SENT)
    _same_bits(got, ref, "cross")


@pytest.mark.parametrize("n,l", [(1000, 130), (700, 1500)])
def test_pair_mma_k64_stages_equal_k32_bits(pcc_gpu, n, l):
    """The pair form with K = 64 stages (three 64 KB stages, 128-byte
    swizzle) issues the same MMAs in the same K order as K = 32 stages, and
    accumulator chunks end at the same samples for both (l = 1,500: three
    chunks), so the results are the same bits."""
    import torch
    pcc = pcc_gpu
    X = torch.from_numpy(_data(n, l, 86 + l)).cuda()
    Z = pcc.pcc_standardize(X, "fp16x3s")
    old = pcc.pcc_get_tuning()
    try:
        pcc.pcc_set_tuning(stage_k=32, cluster=1, pair_mma=0)
        ref = _upper(pcc, Z, n)
        pcc.pcc_set_tuning(stage_k=64, cluster=2, pair_mma=1)
        got = _upper(pcc, Z, n)
    finally:
        pcc.pcc_set_tuning(old["stage_k"], old["cluster"], old["band_rows"],
                           pair_mma=old["pair_mma"])
    assert not np.any(got == SENT)
    _same_bits(got, ref, f"K=64 pair {n}x{l}")
