"""GPU parity: the CUDA path through the C ABI against the FP64 oracle,
element by element, on seeded inputs that span several tiles with ragged
tails, plus the degenerate cases of the method.

Tolerances (max |r_gpu - r_oracle| over non-NaN pairs; NaN sets must be
identical):
  FP64 CUDA-core path      1e-12
  FP32 CUDA-core path      4e-6   (FP32 accumulation over l <= 1024)
  BF16X3 / FP16X3S tensor  1e-5   (the split-precision target)
  BF16X1 tensor            reported only (sanity bound 2e-2)
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 4e-6, "bf16x3": 1e-5, "fp16x3s": 1e-5,
       "bf16x4": 1e-5, "bf16x1": 2e-2}


def _torch():
    import torch
    return torch


def gpu_allpairs(pcc, X, prec, t_ranges=None):
    torch = _torch()
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Z = pcc.pcc_standardize(Xd, prec)
    n = X.shape[0]
    dt = torch.float64 if prec == "fp64" else torch.float32
    R = torch.full((n * (n - 1) // 2,), 7.0, dtype=dt, device="cuda")
    if t_ranges is None:
        pcc.pcc_allpairs_upper(Z, R)
    else:
        for a, b in t_ranges:
            pcc.pcc_allpairs_upper(Z, R, a, b)
    st = pcc.pcc_sync_status(Z)
    assert st == 0, pcc.pcc_status_string(st)
    out = R.cpu().numpy().astype(np.float64)
    return out, Z


def compare(got, want, tol, what=""):
    gn, wn = np.isnan(got), np.isnan(want)
    assert np.array_equal(gn, wn), f"{what}: NaN pattern differs"
    assert not np.any(got == 7.0), f"{what}: unwritten output"
    if (~wn).any():
        err = np.max(np.abs(got[~wn] - want[~wn]))
        assert err <= tol, f"{what}: max|dr| = {err:.3e} > {tol:.1e}"
        return err
    return 0.0


def _data(n, l, seed, kind="counts"):
    if kind == "counts":
        X = synth.counts_log(n, l, seed, dtype=np.float32)
    else:
        X = synth.uniform01(n, l, seed)
    # degenerate rows: a constant row and a huge-offset row
    if n > 4:
        X[n // 3] = 3.25
        X[n // 2] = X[n // 2] + np.float32(1e5)
    return X


SHAPES = [(2, 2), (3, 5), (127, 33), (128, 64), (129, 65), (255, 31),
          (257, 128), (300, 200), (513, 96), (700, 257)]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "fp16x3s",
                                  "bf16x4", "bf16x1"])
@pytest.mark.parametrize("n,l", SHAPES)
def test_allpairs_parity(pcc_gpu, prec, n, l):
    X = _data(n, l, seed=1000 + 7 * n + l)
    if prec == "fp64":
        X = X.astype(np.float64)
    got, _ = gpu_allpairs(pcc_gpu, X, prec)
    want = oracle.pcc_upper(X)
    compare(got, want, TOL[prec], f"{prec} n={n} l={l}")


def test_fp64_modules_config(pcc_gpu):
    """The plain FP64 workload: n=2000, l=128, 8 + N(0,1) with 10 planted
    modules of 50 genes; full packed triangle in FP64."""
    X = synth.modules_normal(2000, 128, seed=1)
    got, _ = gpu_allpairs(pcc_gpu, X, "fp64")
    want = oracle.pcc_upper(X)
    compare(got, want, 1e-12, "fp64 2000x128")


@pytest.mark.parametrize("n,l,prec,tol", [
    (300, 1500, "fp16x3s", 1e-5),   # 3 accumulator chunks (l > 1,024)
    (300, 1500, "bf16x3", 1e-5),
    (257, 2049, "auto", 1e-5),
    (300, 5000, "auto", 1e-5),      # the paper's row length
    # count data shaped like the paper's human dataset (l = 5,072), with
    # planted modules: the default form with a 2x margin on 1e-5
    (640, 5072, "auto", 5e-6),
])
def test_long_rows_parity(pcc_gpu, n, l, prec, tol):
    """Rows past 1,024 samples (each unit accumulated in chunks of at most
    640 samples, every chunk added into the next before the stores)
    against the oracle, with planted modules (r -> 1), a constant row and a
    1e5 offset row."""
    X = _data(n, l, seed=3000 + n + l)
    got, _ = gpu_allpairs(pcc_gpu, X, prec)
    want = oracle.pcc_upper(X)
    err = compare(got, want, tol, f"{prec} n={n} l={l}")
    print(f"{prec} n={n} l={l}: max|dr| {err:.2e}")


class _Knobs:
    """Sets band rows and the CTA-pair form for the block; restores them."""

    def __init__(self, pcc, band, pair):
        self.pcc, self.band, self.pair = pcc, band, pair

    def __enter__(self):
        self.old = self.pcc.pcc_get_tuning()
        self.pcc.pcc_set_tuning(band_rows=self.band,
                                cluster=2 if self.pair else 1,
                                pair_mma=self.pair)

    def __exit__(self, *a):
        o = self.old
        self.pcc.pcc_set_tuning(o["stage_k"], o["cluster"], o["band_rows"],
                                pair_mma=o["pair_mma"])


@pytest.mark.parametrize("n,l", [(4500, 64), (4100, 1100), (4100, 1950)])
@pytest.mark.parametrize("band,pair", [(1, 1), (2, 0)])
def test_steady_state_parity(pcc_gpu, n, l, band, pair):
    """Shapes large enough for the persistent loop's steady state: several
    units per CTA (or CTA pair), many band transitions (one or two
    super-tile rows per band), accumulator buffers reused unit after unit,
    and 2 and 4 accumulator chunks per unit in sequence; every pair
    against the oracle."""
    X = _data(n, l, seed=4000 + n + l)
    with _Knobs(pcc_gpu, band, pair):
        got, Z = gpu_allpairs(pcc_gpu, X, "fp16x3s")
        T = Z.num_tiles()
    # more tiles than workers: each CTA (pair) walks several of them
    assert T > 152
    want = oracle.pcc_upper(X)
    err = compare(got, want, 1e-5, f"n={n} l={l} band={band} pair={pair}")
    print(f"n={n} l={l} band={band} pair={pair}: max|dr| {err:.2e}")


@pytest.mark.parametrize("prec", ["fp16x3s", "bf16x3", "fp32", "fp64"])
def test_near_constant_rows(pcc_gpu, prec):
    """Rows whose mean dwarfs their spread (FP32 input): the row statistics
    must not cancel.  1e7 + N(0, 1e-3) rounds to a constant in FP32 (ulp 1)
    and must be flagged exactly as the oracle's 0/0; 1e4 + N(0, 1e-2) and
    1e6 + N(0, 1) keep a spread of a few FP32 ulps and must match the
    oracle's r; a pair of them is planted as exact affine copies."""
    rng = np.random.default_rng(77)
    n, l = 200, 300
    X = synth.counts_log(n, l, 78, dtype=np.float32)
    base4 = (1e4 + rng.normal(0, 1e-2, l)).astype(np.float32)
    for k in range(10):
        X[k] = (1e7 + rng.normal(0, 1e-3, l)).astype(np.float32)
        X[10 + k] = (1e4 + rng.normal(0, 1e-2, l)).astype(np.float32)
        X[20 + k] = (1e6 + rng.normal(0, 1.0, l)).astype(np.float32)
    X[30] = base4
    X[31] = base4 + np.float32(2.0)  # exact in FP32: r = 1
    Xin = X.astype(np.float64) if prec == "fp64" else X
    got, _ = gpu_allpairs(pcc_gpu, Xin, prec)
    want = oracle.pcc_upper(Xin)
    assert np.isnan(want[pcc_gpu.pcc_pair_index(n, 0, 50)])  # flagged row
    assert not np.isnan(want[pcc_gpu.pcc_pair_index(n, 10, 50)])
    compare(got, want, TOL[prec], f"{prec} near-constant rows")


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3s"])
def test_perfect_correlation_rows(pcc_gpu, prec):
    """|r| -> 1 is where the dropped lo*lo term peaks: rows that are exact
    affine copies of each other (r = +-1) and a Hadamard block (r = 0)."""
    rng = np.random.default_rng(3)
    base = rng.standard_normal(256).astype(np.float32)
    rows = [base * a + b for a, b in [(1, 0), (2, 5), (-3, 1), (0.5, -9)]]
    H = np.array([[1.0]])
    for _ in range(8):
        H = np.block([[H, H], [H, -H]])
    X = np.vstack(rows + [H[1:300].astype(np.float32)]).astype(np.float32)
    got, _ = gpu_allpairs(pcc_gpu, X, prec)
    want = oracle.pcc_upper(X)
    compare(got, want, 1e-5, prec)


@pytest.mark.parametrize("prec", ["fp32", "fp16x3s"])
def test_tile_ranges_union_is_whole(pcc_gpu, prec):
    """Equal tile-id ranges (Section III-D's distribution) computed by
    separate calls cover the triangle exactly once."""
    X = _data(900, 70, seed=5)
    whole, Z = gpu_allpairs(pcc_gpu, X, prec)
    T = Z.num_tiles()
    for parts in (2, 3, 7):
        step = -(-T // parts)
        ranges = [(min(i * step, T), min((i + 1) * step, T))
                  for i in range(parts)]
        got, _ = gpu_allpairs(pcc_gpu, X, prec, ranges)
        assert np.array_equal(np.isnan(got), np.isnan(whole))
        ok = ~np.isnan(whole)
        assert np.array_equal(got[ok], whole[ok])


def test_standardize_forms(pcc_gpu):
    """K1 against Eq. (5) computed by the oracle, for every stored form."""
    torch = _torch()
    for n, l in [(3, 2), (129, 65), (1000, 300)]:
        X = _data(n, l, seed=n + l)
        Zo, fo = oracle.standardize(X)
        Xd = torch.from_numpy(X).cuda()
        for prec in ["fp64", "fp32", "bf16x3", "fp16x3s", "bf16x4",
                     "bf16x1"]:
            Z = pcc_gpu.pcc_standardize(Xd, prec)
            info = Z.info()
            buf = Z.buffers()
            lpad = info["lpad"]
            assert lpad % 64 == 0 and lpad >= l
            fl = torch.empty(n, dtype=torch.uint8, device="cuda")
            _copy_from_ptr(fl, buf["flags"])
            assert np.array_equal(fl.cpu().numpy(), fo), prec
            if prec in ("fp64", "fp32"):
                dt = torch.float64 if prec == "fp64" else torch.float32
                z = torch.empty((n, lpad), dtype=dt, device="cuda")
                _copy_from_ptr(z, buf["z"])
                z = z.cpu().numpy().astype(np.float64)
                tol = 1e-15 if prec == "fp64" else 3e-7
            else:
                dt = torch.float16 if prec == "fp16x3s" else torch.bfloat16
                hi = torch.empty((n, lpad), dtype=dt, device="cuda")
                _copy_from_ptr(hi, buf["hi"])
                z = hi.float().cpu().numpy().astype(np.float64)
                if buf["lo"]:
                    lo = torch.empty((n, lpad), dtype=dt, device="cuda")
                    _copy_from_ptr(lo, buf["lo"])
                    z = z + lo.float().cpu().numpy().astype(np.float64)
                z = z * 2.0 ** (-info["scale_exp"])
                tol = {"bf16x3": 2e-5, "fp16x3s": 4e-7, "bf16x4": 2e-5,
                       "bf16x1": 4e-3}[prec]
            assert np.all(z[:, l:] == 0), prec
            err = np.max(np.abs(z[:, :l] - Zo))
            assert err <= tol, (prec, n, l, err)
            Z.close()


@pytest.mark.parametrize("l", [7, 100, 128, 200, 256, 500, 512])
def test_standardize_row_pitch_gives_same_bits(pcc_gpu, l):
    """16-byte aligned rows are read with float4 loads, rows with an odd
    pitch with scalar loads; both sum in the same order, so the stored
    halves and flags are the same bits (FP16X3S, BF16X3, FP32)."""
    torch = _torch()
    n = 333
    X = _data(n, l, seed=40 + l)
    wide = np.zeros((n, l + 1), dtype=np.float32)
    wide[:, :l] = X
    Xa = torch.from_numpy(X).cuda()                 # pitch l (aligned if 4 | l)
    Xu = torch.from_numpy(wide).cuda()[:, :l]       # pitch l + 1
    for prec in ("fp16x3s", "bf16x3", "fp32"):
        za = pcc_gpu.pcc_standardize(Xa, prec)
        zu = pcc_gpu.pcc_standardize(Xu, prec)
        lpad = za.info()["lpad"]
        ba, bu = za.buffers(), zu.buffers()
        for key in ("hi", "lo", "z"):
            if not ba[key]:
                continue
            bytes_per = 4 if key == "z" else 2
            a = torch.empty(n * lpad * bytes_per, dtype=torch.uint8,
                            device="cuda")
            u = torch.empty_like(a)
            _copy_from_ptr(a, ba[key])
            _copy_from_ptr(u, bu[key])
            assert torch.equal(a, u), (prec, key, l)
        fa = torch.empty(n, dtype=torch.uint8, device="cuda")
        fu = torch.empty_like(fa)
        _copy_from_ptr(fa, ba["flags"])
        _copy_from_ptr(fu, bu["flags"])
        assert torch.equal(fa, fu)
        za.close()
        zu.close()


def _copy_from_ptr(dst, ptr):
    """Device-to-device copy from a raw library-owned pointer (driver API,
    unified addressing)."""
    import ctypes
    torch = _torch()
    torch.cuda.synchronize()
    libcuda = ctypes.CDLL("libcuda.so.1")
    nbytes = dst.numel() * dst.element_size()
    res = libcuda.cuMemcpy(ctypes.c_uint64(dst.data_ptr()),
                           ctypes.c_uint64(ptr), ctypes.c_size_t(nbytes))
    assert int(res) == 0
    torch.cuda.synchronize()


def _edges_gpu(pcc, X, prec, tau, cap=1 << 20, with_R=True):
    torch = _torch()
    Xd = torch.from_numpy(X).cuda()
    Z = pcc.pcc_standardize(Xd, prec)
    n = X.shape[0]
    R = (torch.full((n * (n - 1) // 2,), 7.0, device="cuda")
         if with_R else None)
    E = torch.zeros(cap * pcc.EDGE_BYTES, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    pcc.pcc_threshold_edges(Z, tau, E, cap, cnt, R)
    st = pcc.pcc_sync_status(Z)
    c = int(cnt.item())
    i, j, r = pcc.edges_view(E, min(c, cap))
    return Z, st, c, (i, j, r), (None if R is None else R.cpu().numpy())


def check_edges_band(X, tau, gi, gj, gr, band=1e-5, i0=0, i1=None):
    """The GPU edge set equals the oracle's outside |(|r| - tau)| <= band;
    inside the band either answer is accepted."""
    n = X.shape[0]
    oi, oj, orr = oracle.edges(X, tau, i0, i1 if i1 is not None else n)
    want = set(zip(oi.tolist(), oj.tolist()))
    got = set(zip(gi.tolist(), gj.tolist()))
    assert len(got) == len(gi), "duplicate edges"
    for a, b in got - want:
        r = oracle.pcc_pairs(X, [a], [b])[0]
        assert abs(abs(r) - tau) <= band, ("extra edge", a, b, r)
    for a, b in want - got:
        r = oracle.pcc_pairs(X, [a], [b])[0]
        assert abs(abs(r) - tau) <= band, ("missing edge", a, b, r)
    if len(gi):
        ref = oracle.pcc_pairs(X, gi, gj)
        assert np.max(np.abs(ref - gr)) <= 1e-5
    return len(want)


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3s", "fp32"])
def test_threshold_edges(pcc_gpu, prec):
    X = synth.counts_log(1500, 150, seed=77)
    X[10] = 1.0  # a flagged row never makes an edge
    Z, st, c, (i, j, r), R = _edges_gpu(pcc_gpu, X, prec, 0.8)
    assert st == 0
    assert np.all(i < j)
    k = check_edges_band(X, 0.8, i, j, r)
    assert k > 100  # the planted modules give many edges
    # the packed output written in the same pass equals allpairs_upper
    whole, _ = gpu_allpairs(pcc_gpu, X, prec)
    assert np.array_equal(np.isnan(R), np.isnan(whole))
    ok = ~np.isnan(whole)
    assert np.array_equal(R[ok].astype(np.float64), whole[ok])


def test_threshold_edges_capacity(pcc_gpu):
    X = synth.counts_log(1500, 150, seed=77)
    Z, st, c, (i, j, r), _ = _edges_gpu(pcc_gpu, X, "fp16x3s", 0.5, cap=64,
                                        with_R=False)
    assert c > 64
    assert st == pcc_gpu.PCC_ERR_CAPACITY
    assert len(i) == 64 and np.all(i < j)
    ref = oracle.pcc_pairs(X, i, j)
    assert np.all(np.abs(ref) >= 0.5 - 1e-5)
    # the count is the true total
    oi, _, _ = oracle.edges(X, 0.5)
    assert abs(c - len(oi)) <= 5


def test_invalid_arguments(pcc_gpu):
    torch = _torch()
    X = torch.zeros((1, 8), device="cuda")
    with pytest.raises(pcc_gpu.PccError):
        pcc_gpu.pcc_standardize(X, "fp16x3s")
    X = torch.randn((10, 8), device="cuda")
    Z = pcc_gpu.pcc_standardize(X, "fp16x3s")
    R = torch.empty(45, device="cuda")
    with pytest.raises(pcc_gpu.PccError):
        pcc_gpu.pcc_allpairs_upper(Z, R, 0, Z.num_tiles() + 1)
    with pytest.raises(pcc_gpu.PccError):
        pcc_gpu.pcc_allpairs_upper(Z, R.double())


def test_sharded_ranks_cover_the_triangle(pcc_gpu):
    """Section III-D's equal tile ranges, one call per (simulated) rank into
    the same output: every pair is written exactly by its owner."""
    from paper_1605_01584_gb300 import shard
    torch = _torch()
    X = _data(1500, 96, seed=8)
    whole, Z = gpu_allpairs(pcc_gpu, X, "auto")
    R = torch.full((1500 * 1499 // 2,), 7.0, device="cuda")
    covered = 0
    for rank in range(3):
        b, e = shard.allpairs_sharded(Z, R, rank, 3)
        covered += e - b
    assert covered == Z.num_tiles()
    got = R.cpu().numpy().astype(np.float64)
    assert not np.any(got == 7.0)
    assert np.array_equal(np.isnan(got), np.isnan(whole))
    ok = ~np.isnan(whole)
    assert np.array_equal(got[ok], whole[ok])
