"""Host-memory entry points: pcc_standardize_host copies a host matrix in
and standardizes it exactly as pcc_standardize does from device memory;
pcc_edges_copy_host brings an edge list and its count back."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _bits(a):
    return a.view(np.uint32)


@pytest.mark.parametrize("prec,pad,pinned", [("fp16x3s", 0, True),
                                             ("bf16x3", 3, False),
                                             ("fp64", 0, True)])
def test_standardize_host_equals_device_input(pcc_gpu, prec, pad, pinned):
    import torch
    pcc = pcc_gpu
    n, l = 1100, 150
    X = synth.counts_log(n, l, 91)
    X[7] = 2.0  # flagged
    if prec == "fp64":
        X = X.astype(np.float64)
    W = np.zeros((n, l + pad), dtype=X.dtype)
    W[:, :l] = X
    Wh = torch.from_numpy(W)
    if pinned:
        Wh = Wh.pin_memory()
    Xh = Wh[:, :l]
    dt = torch.float64 if prec == "fp64" else torch.float32
    Zd = pcc.pcc_standardize(torch.from_numpy(X).cuda(), prec)
    Zh = pcc.pcc_standardize_host(Xh, prec)
    Zh2 = pcc.pcc_standardize_host(Xh, prec, Z=Zh)  # reused in place
    assert Zh2 is Zh
    out = []
    for Z in (Zd, Zh):
        R = torch.full((n * (n - 1) // 2,), 7.0, dtype=dt, device="cuda")
        pcc.pcc_allpairs_upper(Z, R)
        assert pcc.pcc_sync_status(Z) == 0
        out.append(R.cpu().numpy())
    a, b = out
    assert np.array_equal(np.isnan(a), np.isnan(b))
    ok = ~np.isnan(a)
    assert np.array_equal(a[ok].view(np.uint8), b[ok].view(np.uint8))


def test_edges_copy_host(pcc_gpu):
    import torch
    pcc = pcc_gpu
    n, l = 1500, 64
    X = torch.from_numpy(synth.counts_log(n, l, 92)).cuda()
    Z = pcc.pcc_standardize(X, "fp16x3s")
    cap = 1 << 16
    E = torch.zeros(cap * pcc.EDGE_BYTES, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    pcc.pcc_threshold_edges(Z, 0.5, E, cap, cnt, None)
    Eh = torch.zeros(cap * pcc.EDGE_BYTES, dtype=torch.uint8)
    c = pcc.pcc_edges_copy_host(E, cnt, cap, Eh)
    assert c == int(cnt.item()) and 0 < c <= cap
    assert torch.equal(Eh[:c * pcc.EDGE_BYTES].cuda(),
                       E[:c * pcc.EDGE_BYTES])
    # a host array smaller than the count: the records that fit are copied
    # and the overflow is reported
    small = max(1, c // 2)
    Es = torch.zeros(small * pcc.EDGE_BYTES, dtype=torch.uint8)
    with pytest.raises(pcc.PccError) as e:
        pcc.pcc_edges_copy_host(E, cnt, small, Es)
    assert e.value.status == pcc.PCC_ERR_CAPACITY
    assert torch.equal(Es.cuda(), E[:small * pcc.EDGE_BYTES])
