"""The autotuner times every candidate on the same trajectory, requires them to agree on
the final state (the trajectory does not depend on the kernel or its tuning, Sec. 3),
and caches the fastest per size class."""
import json

import pytest

pytestmark = pytest.mark.gpu

ac = pytest.importorskip("paper_cs_0502039_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_cs_0502039_gb300 import autotune  # noqa: E402


def test_tune_small_class(tmp_path):
    path = str(tmp_path / "tune.json")
    entry = autotune.tune(200, 180, T=1.0, cache_path=path)
    assert entry["kernel"] in (ac.AC_KERNEL_ROUND, ac.AC_KERNEL_BLOCKED, ac.AC_KERNEL_EPOCH)
    assert entry["events_per_s"] > 0 and len(entry["measured"]) == len(autotune.CANDIDATES)
    cached = json.load(open(path))
    assert autotune.class_key(200, 180) in cached
    assert autotune.tune(256, 256, cache_path=path) == entry      # same class: served from the cache
    with ac.Sim(200, 180, 0.44, 1.0, 0.0, 3) as sim:
        autotune.apply(sim, entry)
        sim.run_until(1)


def test_beta_buckets_are_separate_classes(tmp_path):
    path = str(tmp_path / "tune.json")
    few = [c for c in autotune.CANDIDATES if c["kernel"] != ac.AC_KERNEL_BLOCKED][:3]
    hot = autotune.tune(128, 128, T=1.0, cache_path=path, beta=0.3, candidates=few)
    cold = autotune.tune(128, 128, T=1.0, cache_path=path, beta=0.6, candidates=few)
    cached = json.load(open(path))
    assert autotune.class_key(128, 128, 0.3) in cached and autotune.class_key(128, 128, 0.6) in cached
    assert len(hot["measured"]) == len(cold["measured"]) == 3


def test_tune_batch_agrees_on_every_lattice(tmp_path):
    """Every batch candidate must reach the same per-lattice fingerprints (the batch runs
    inside tune_batch raise otherwise); the choice is cached per batch class."""
    path = str(tmp_path / "tune.json")
    lats = [(64, 64, 0.3), (96, 130, 0.44), (200, 180, 0.6), (40, 72, 0.5)]
    entry = autotune.tune_batch(lats, T=1.0, cache_path=path)
    assert entry["kernel"] in (ac.AC_KERNEL_ROUND, ac.AC_KERNEL_EPOCH)
    assert len(entry["measured"]) == len(autotune.BATCH_CANDIDATES)
    assert autotune.batch_key(lats) in json.load(open(path))
    only = autotune.tune_batch(lats, T=1.0, cache_path=path, batched_only=True)
    assert only["batched"] and len(only["measured"]) == sum(c["batched"] for c in autotune.BATCH_CANDIDATES)
