"""Host logic of the autotuner (no GPU): the crossover choice and the JSON cache."""
from paper_1502_07770_gb300 import autotune


def test_crossover_choice():
    t = {(512, 256): (1.0, 2.0), (512, 1024): (1.0, 2.0),
         (1024, 256): (1.0, 1.5), (1024, 1024): (1.0, 1.2),
         (2048, 256): (1.0, 0.9), (2048, 1024): (1.0, 1.1),
         (4096, 256): (2.0, 1.0), (4096, 1024): (2.0, 1.0)}
    # the warp kernel must win for every length: 2048 fails at n = 256
    assert autotune.choose_crossover(t) == 1024
    assert autotune.choose_crossover({(512, 256): (3.0, 1.0)}) == 0


def test_cache_roundtrip(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert autotune.load_cache(path) == {}
    autotune.save_cache({"GPU|tv100": {"coop_max_chains": 2048, "batched_warps": 4}}, path)
    assert autotune.load_cache(path)["GPU|tv100"]["batched_warps"] == 4
