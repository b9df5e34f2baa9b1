"""The tuner's cache logic (CPU) and one small tuning run (GPU)."""
import numpy as np
import pytest

from paper_1605_01584_gb300 import autotune


def test_bucket_and_nearest_lookup(tmp_path):
    p = str(tmp_path / "t.json")
    assert autotune.bucket(65536, 512, "bf16x3") == "n65536_l512_bf16x3"
    assert autotune.bucket(50000, 500, "bf16x3") == "n65536_l512_bf16x3"
    assert autotune.bucket(40000, 33, "fp16x3s") == "n32768_l64_fp16x3s"
    cache = {
        "n16384_l512_bf16x3": {"best": {"stage_k": 64, "cluster": 1,
                                        "band_rows": 16}},
        "n65536_l512_bf16x3": {"best": {"stage_k": 32, "cluster": 2,
                                        "band_rows": 32}},
    }
    autotune.save_cache(cache, p)
    c = autotune.load_cache(p)
    assert c == cache
    assert autotune.lookup(65536, 512, "bf16x3", c)["stage_k"] == 32
    assert autotune.lookup(20000, 512, "bf16x3", c)["stage_k"] == 64
    assert autotune.lookup(20000, 1024, "bf16x3", c) is None
    assert autotune.load_cache(str(tmp_path / "missing.json")) == {}


@pytest.mark.gpu
def test_tune_small_shape_and_apply(pcc_gpu, tmp_path):
    import torch
    pcc = pcc_gpu
    p = str(tmp_path / "tune.json")
    before = pcc.pcc_get_tuning()
    e = autotune.tune_pairs(2048, 128, "bf16x3", reps=2, path=p,
                            candidates={"band_rows": (8, 32)})
    # K = 32 or 64 stages x CTA pairs or single CTAs x two band heights
    assert len(e["all"]) == 8 and e["best"]["ms"] > 0
    assert pcc.pcc_get_tuning() == before  # tuning run restores the knobs
    X = torch.rand((2048, 128), device="cuda")
    Z = pcc.pcc_standardize(X, "bf16x3")
    R0 = torch.empty(2048 * 2047 // 2, device="cuda")
    pcc.pcc_allpairs_upper(Z, R0)
    try:
        assert autotune.apply(2048, 128, "bf16x3",
                              autotune.load_cache(p))
        R1 = torch.empty_like(R0)
        pcc.pcc_allpairs_upper(Z, R1)
        torch.cuda.synchronize()
        assert torch.equal(R0, R1)  # knobs never change results
    finally:
        pcc.pcc_set_tuning(before["stage_k"], before["cluster"],
                           before["band_rows"], pair_mma=before["pair_mma"])


def test_lookup_skips_unusable_entries():
    good = {"best": {"stage_k": 32, "cluster": 2, "band_rows": 32}}
    cache = {
        "n65536_l512_bf16x3": {"runs": []},                 # no 'best'
        "n32768_l512_bf16x3": {"best": {"stage_k": 64}},    # knobs missing
        "n16384_l512_bf16x3": good,
        "n8192_l512_bf16x3": "garbage",
    }
    # the exact bucket and the nearer entry are unusable: the usable one
    # further away is taken
    assert autotune.lookup(65536, 512, "bf16x3", cache) == good["best"]
    assert autotune.lookup(65536, 512, "fp16x3s", cache) is None
    assert autotune.lookup(65536, 512, "bf16x3", {}) is None


def test_lookup_batched_takes_the_best_run_of_the_stage_size():
    runs = [{"stage_k": 64, "cluster": 1, "pair_mma": 0, "band_rows": 8,
             "ms": 1.0},
            {"stage_k": 32, "cluster": 1, "pair_mma": 0, "band_rows": 16,
             "ms": 1.2},
            {"stage_k": 32, "cluster": 2, "pair_mma": 1, "band_rows": 32,
             "ms": 1.1}]
    cache = {"n4096_l512_fp16x3s": {"best": runs[0], "all": runs}}
    lb = autotune.lookup_batched
    assert lb(4096, 500, "fp16x3s", cache, stage_k=32) == (1, 32)
    assert lb(4096, 500, "fp16x3s", cache, stage_k=64) == (0, 8)
    # nearest n in the same (padded l, form) bucket
    assert lb(3000, 512, "fp16x3s", cache, stage_k=32) == (1, 32)
    assert lb(4096, 700, "fp16x3s", cache, stage_k=32) is None
    cache["n4096_l512_fp16x3s"]["all"] = runs[:1]  # no K = 32 run
    assert lb(4096, 512, "fp16x3s", cache, stage_k=32) is None
