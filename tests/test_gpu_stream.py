"""Outputs delivered to host memory in overlapped passes (Section III-C's
multi-pass execution, Algorithm 2): the packed triangle and the dense cross
matrix, computed a run of row blocks at a time into two device windows.

Every pass runs the same kernels on the same tiles as the one-shot call, so
the host result must equal the device result bit for bit; the oracle checks
the one-shot call elsewhere, and once more here on the streamed values.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 4e-6, "bf16x3": 1e-5, "fp16x3s": 1e-5}


def _z(pcc, X, prec):
    import torch
    return pcc.pcc_standardize(torch.from_numpy(X).cuda(), prec)


def _device_upper(pcc, Z, n, f64=False):
    import torch
    R = torch.full((n * (n - 1) // 2,), 7.0, device="cuda",
                   dtype=torch.float64 if f64 else torch.float32)
    pcc.pcc_allpairs_upper(Z, R)
    assert pcc.pcc_sync_status(Z) == 0
    return R.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "fp16x3s"])
def test_upper_host_equals_device_bits(pcc_gpu, prec):
    pcc = pcc_gpu
    n, l = 1500, 72
    X = synth.counts_log(n, l, 21, dtype=np.float32)
    X[7] = 1.0
    if prec == "fp64":
        X = X.astype(np.float64)
    Z = _z(pcc, X, prec)
    f64 = prec == "fp64"
    want = _device_upper(pcc, Z, n, f64)
    npairs = n * (n - 1) // 2
    H = np.full(npairs, 7.0, dtype=np.float64 if f64 else np.float32)
    seen = []
    # a budget of a few row blocks: many passes
    pcc.pcc_allpairs_upper_host(Z, H, device_bytes=3 << 20,
                                sink=lambda a, b, v: seen.append((a, b)))
    assert pcc.pcc_sync_status(Z) == 0
    assert len(seen) >= 3
    assert seen[0][0] == 0 and seen[-1][1] == n
    assert all(b0 == a1 for (_, b0), (a1, _) in zip(seen, seen[1:]))
    assert np.array_equal(np.isnan(H), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.array_equal(H[ok], want[ok])
    ref = oracle.pcc_upper(X)
    assert np.nanmax(np.abs(H.astype(np.float64) - ref)) <= TOL[prec]


def test_upper_staged_sink_slices(pcc_gpu):
    """No host triangle: each packed slice arrives in a staging buffer."""
    pcc = pcc_gpu
    n, l = 1300, 40
    X = synth.counts_log(n, l, 22, dtype=np.float32)
    Z = _z(pcc, X, "bf16x3")
    want = _device_upper(pcc, Z, n)
    parts = []
    pcc.pcc_allpairs_upper_host(
        Z, None, device_bytes=4 << 20,
        sink=lambda a, b, v: parts.append((a, b, v.copy())))
    assert len(parts) >= 3
    got = np.concatenate([v for _, _, v in parts])
    assert got.size == want.size
    ok = ~np.isnan(want)
    assert np.array_equal(got[ok], want[ok])
    for a, b, v in parts:
        assert v.size == (b * (2 * n - b - 1) - a * (2 * n - a - 1)) // 2


def test_sink_abort_and_recovery(pcc_gpu):
    pcc = pcc_gpu
    n = 1200
    X = synth.counts_log(n, 48, 23, dtype=np.float32)
    Z = _z(pcc, X, "fp16x3s")
    calls = []

    def sink(a, b, v):
        calls.append(a)
        if len(calls) == 2:
            raise KeyboardInterrupt("stop")

    with pytest.raises(KeyboardInterrupt):
        pcc.pcc_allpairs_upper_host(Z, None, device_bytes=4 << 20, sink=sink)
    assert len(calls) == 2
    # the library and the device are still usable
    H = np.empty(n * (n - 1) // 2, dtype=np.float32)
    pcc.pcc_allpairs_upper_host(Z, H, device_bytes=4 << 20)
    want = _device_upper(pcc, Z, n)
    assert np.array_equal(H, want, equal_nan=True)


def test_budget_too_small_is_an_error(pcc_gpu):
    pcc = pcc_gpu
    n = 2000
    X = synth.counts_log(n, 32, 24, dtype=np.float32)
    Z = _z(pcc, X, "bf16x3")
    H = np.empty(n * (n - 1) // 2, dtype=np.float32)
    with pytest.raises(pcc.PccError) as ei:
        pcc.pcc_allpairs_upper_host(Z, H, device_bytes=1 << 16)
    assert ei.value.status == pcc.PCC_ERR_OOM
    with pytest.raises(pcc.PccError):
        pcc.pcc_allpairs_upper_host(Z, None)  # neither host buffer nor sink


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_cross_host_pitch(pcc_gpu, prec):
    import torch
    pcc = pcc_gpu
    nx, ny, l = 1100, 700, 56
    X = synth.counts_log(nx, l, 25, dtype=np.float32)
    Y = synth.counts_log(ny, l, 26, dtype=np.float32)
    ZX, ZY = _z(pcc, X, prec), _z(pcc, Y, prec)
    Rd = torch.full((nx, ny), 7.0, device="cuda")
    pcc.pcc_cross_allpairs(ZX, ZY, Rd)
    assert pcc.pcc_sync_status(ZX) == 0
    want = Rd.cpu().numpy()
    H = np.full((nx, ny + 9), 7.0, dtype=np.float32)
    rows = []
    pcc.pcc_cross_allpairs_host(ZX, ZY, H, device_bytes=2 << 20,
                                sink=lambda a, b, v: rows.append((a, b)))
    assert len(rows) >= 3 and rows[-1][1] == nx
    assert np.all(H[:, ny:] == 7.0)
    assert np.array_equal(H[:, :ny], want, equal_nan=True)
    ref = oracle.cross_rows(X, Y)
    assert np.nanmax(np.abs(H[:, :ny] - ref)) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "fp16x3s"])
def test_threshold_edges_host_matches_device_call(pcc_gpu, prec):
    """Edges and the host triangle from the passes equal one device call:
    the same edge set (order aside) and the same R bits."""
    import torch
    pcc = pcc_gpu
    n, l, tau = 1400, 64, 0.6
    X = synth.counts_log(n, l, 27, dtype=np.float32)
    Z = _z(pcc, X, prec)
    cap = 1 << 18
    E1 = torch.zeros(cap * 12, dtype=torch.uint8, device="cuda")
    E2 = torch.zeros_like(E1)
    c1 = torch.zeros(1, dtype=torch.int64, device="cuda")
    c2 = torch.zeros_like(c1)
    R1 = torch.full((n * (n - 1) // 2,), 7.0, device="cuda")
    pcc.pcc_threshold_edges(Z, tau, E1, cap, c1, R1)
    H = np.full(n * (n - 1) // 2, 7.0, dtype=np.float32)
    passes = []
    pcc.pcc_threshold_edges_host(Z, tau, E2, cap, c2, H,
                                 device_bytes=3 << 20,
                                 sink=lambda a, b, v: passes.append(a))
    assert pcc.pcc_sync_status(Z) == 0
    assert len(passes) >= 3
    k1, k2 = int(c1.item()), int(c2.item())
    assert k1 == k2 and k1 > 100
    def edge_set(E, k):
        rec = E[:k * 12].cpu().numpy().view(np.uint32).reshape(-1, 3)
        return set(map(tuple, rec.tolist()))
    assert edge_set(E1, k1) == edge_set(E2, k2)
    assert np.array_equal(H, R1.cpu().numpy(), equal_nan=True)
