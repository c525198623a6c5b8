"""Host logic of the autotuner: class keys and temperature buckets (no GPU needed)."""
from paper_cs_0502039_gb300 import autotune


def test_beta_buckets():
    assert autotune.beta_bucket(0.25) == 0.30 and autotune.beta_bucket(0.3499) == 0.30
    assert autotune.beta_bucket(0.35) == 0.44 and autotune.beta_bucket(0.4407) == 0.44
    assert autotune.beta_bucket(0.5) == 0.60 and autotune.beta_bucket(3.0) == 0.60


def test_class_keys():
    a = autotune.class_key(4096, 4096, 0.30)
    b = autotune.class_key(4000, 3000, 0.31)
    c = autotune.class_key(4096, 4096, 0.60)
    assert a == b and a != c
    assert autotune.class_key(100, 100) == autotune.class_key(128, 65)


def test_batch_keys():
    lats = [(64, 64, 0.3), (128, 128, 0.5)]
    assert autotune.batch_key(lats) == autotune.batch_key(list(reversed(lats)))
    assert autotune.batch_key(lats) != autotune.batch_key(lats + [(64, 64, 0.4)])
    assert "|batch2|" in autotune.batch_key(lats)
