"""The seeded generators are deterministic and produce the stated shapes."""
import numpy as np

import synth


def test_deterministic_and_shapes():
    a = synth.counts_log(500, 64, seed=7)
    b = synth.counts_log(500, 64, seed=7)
    assert a.shape == (500, 64) and a.dtype == np.float32
    assert np.array_equal(a, b)
    assert not np.array_equal(a, synth.counts_log(500, 64, seed=8))
    x = synth.modules_normal(200, 32, seed=1)
    assert x.shape == (200, 32) and x.dtype == np.float64


def test_fisher_yates_perms_are_permutations():
    p = synth.fisher_yates_perms(64, 37, seed=4)
    assert p.shape == (64, 37) and p.dtype == np.int32
    assert np.all(np.sort(p, axis=1) == np.arange(37))
    assert len({tuple(r) for r in p}) == 64
    assert np.array_equal(p, synth.fisher_yates_perms(64, 37, seed=4))


def test_splitmix64_reference_values():
    # SplitMix64 from state 0: published first output 0xE220A8397B1DCDAF
    st, out = synth.splitmix64(np.array([0], dtype=np.uint64))
    assert int(out[0]) == 0xE220A8397B1DCDAF


def test_uneven_shapes_ranges():
    s = synth.uneven_shapes()
    assert len(s) == 64
    assert all(500 <= n <= 20000 and 32 <= l <= 2048 for n, l in s)


def test_counts_log_many_equals_serial_calls():
    shapes = [(90, 17), (200, 33), (81, 64)]
    seeds = [7, 8, 9]
    got = synth.counts_log_many(shapes, seeds, return_modules=True,
                                workers=2)
    for (n, l), s, (X, mod) in zip(shapes, seeds, got):
        X0, mod0 = synth.counts_log(n, l, s, return_modules=True)
        assert X.dtype == X0.dtype and X.shape == (n, l)
        assert np.array_equal(X.view(np.uint32), X0.view(np.uint32))
        assert np.array_equal(mod, mod0)
    assert [x.shape for x in synth.counts_log_many(shapes[:1], [7])] == \
        [(90, 17)]
