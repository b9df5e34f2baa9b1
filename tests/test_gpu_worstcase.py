"""The split forms at their worst: exact affine copies of rows whose mass
sits in one sample, so that r = +-1 and no error averages out over k.

For such a pair the tensor-core r deviates from the oracle by at most
  (representation) 2 e_z   -- z = hi + lo + e with |e| <= e_z |z|, twice
  (dropped term)   e_z     -- sum lo_i lo_j <= e_z
  (accumulation)   U 2^-22 -- the FP32 accumulator drops up to two ulps of
                              a partial sum <= 1 toward zero at each of its U
                              updates (3 products x chunk/16 instructions:
                              rows longer than 1,024 samples accumulate in
                              chunks of at most 640 samples)
  (folds)          C 2^-24 -- one round-to-nearest add per further chunk
with e_z = 2^-18 for BF16 halves (8-bit significands: |lo| <= 2^-9 |z|, and
lo itself rounded to 8 bits) and 2^-22 for FP16 halves of z 2^s (11-bit
significands).

The default form (AUTO = FP16X3S) must stay within the split form's 1e-5
at every row length up to the paper's l = 5,000.  BF16X3 and BF16X4 are
held to the derived bound, which at every l lies above 1e-5 (their BF16
halves alone give 3 e_z = 1.1e-5), and reported.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

E_Z = {"bf16x3": 2.0 ** -18, "fp16x3s": 2.0 ** -22, "bf16x4": 2.0 ** -18}
# BF16X4 keeps the lo.lo product: one e_z less, one update per K step more
DROPPED = {"bf16x3": 1, "fp16x3s": 1, "bf16x4": 0}
NPROD = {"bf16x3": 3, "fp16x3s": 3, "bf16x4": 4}
ONE_ACC, CHUNK = 1024, 640  # the library's accumulator chunk rule


def _concentrated_copies(l, pairs, seed):
    rng = np.random.default_rng(seed)
    rows = []
    for p in range(pairs):
        x = rng.uniform(0, 0.05, l)
        x[rng.integers(l)] = rng.uniform(20, 60)
        a = [1.0, -2.0, 3.0, -0.5][p % 4]
        rows += [x, a * x + rng.uniform(-5, 5)]
    return np.array(rows, dtype=np.float32)


def _chunks(lpad):
    """Accumulator chunks of a unit (as the library cuts them)."""
    if lpad <= ONE_ACC:
        return 1
    return max(2, -(-lpad // CHUNK))


def _run(pcc, X, prec):
    import torch
    n = X.shape[0]
    Z = pcc.pcc_standardize(torch.from_numpy(X).cuda(), prec)
    R = torch.full((n * (n - 1) // 2,), 7.0, device="cuda")
    pcc.pcc_allpairs_upper(Z, R)
    assert pcc.pcc_sync_status(Z) == 0
    got = R.cpu().numpy().astype(np.float64)
    want = oracle.pcc_upper(X)
    I, J = np.triu_indices(n, 1)
    copies = (J == I + 1) & (I % 2 == 0)
    assert np.all(np.abs(want[copies]) > 1 - 1e-9)
    return got, want, copies, Z.info()


@pytest.mark.parametrize("l", [64, 512, 1024, 2048, 3072, 5000])
def test_default_form_within_1e5_on_exact_copies(pcc_gpu, l):
    X = _concentrated_copies(l, 96, 40 + l)
    got, want, copies, info = _run(pcc_gpu, X, "auto")
    assert info["prec"] == pcc_gpu.PCC_PREC_FP16X3S
    err_copy = np.max(np.abs(got[copies] - want[copies]))
    err_all = np.max(np.abs(got - want))
    print(f"auto l={l} ({_chunks(info['lpad'])} chunks): copies max|dr| "
          f"{err_copy:.2e}, all {err_all:.2e}")
    assert err_all <= 1e-5


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x4"])
@pytest.mark.parametrize("l", [64, 512, 2048, 5000])
def test_bf16_forms_within_derived_bound(pcc_gpu, prec, l):
    X = _concentrated_copies(l, 96, 40 + l)
    got, want, copies, info = _run(pcc_gpu, X, prec)
    lpad = info["lpad"]
    nch = _chunks(lpad)
    per_chunk = -(-(lpad // 32) // nch) * 32  # longest chunk, in samples
    updates = NPROD[prec] * per_chunk // 16
    bound = ((2 + DROPPED[prec]) * E_Z[prec] + updates * 2.0 ** -22 +
             nch * 2.0 ** -24)
    err_copy = np.max(np.abs(got[copies] - want[copies]))
    err_all = np.max(np.abs(got - want))
    print(f"{prec} l={l}: copies max|dr| {err_copy:.2e}, all {err_all:.2e},"
          f" bound {bound:.2e}")
    assert err_all <= bound
