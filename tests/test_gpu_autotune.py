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
    assert entry["kernel"] in (ac.AC_KERNEL_ROUND, ac.AC_KERNEL_BLOCKED)
    assert entry["events_per_s"] > 0 and len(entry["measured"]) == len(autotune.CANDIDATES)
    cached = json.load(open(path))
    assert autotune.class_key(200, 180) in cached
    assert autotune.tune(256, 256, cache_path=path) == entry      # same class: served from the cache
    with ac.Sim(200, 180, 0.44, 1.0, 0.0, 3) as sim:
        autotune.apply(sim, entry)
        sim.run_until(1)
