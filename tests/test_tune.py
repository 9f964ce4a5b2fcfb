"""Autotuner: cache keys and storage (CPU), and on the GPU that a tuned
configuration is valid and changes nothing in the results."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1510_08982_gb300 import inputs


def test_size_class_key_is_stable_under_sampling(monkeypatch, tmp_path):
    from paper_1510_08982_gb300 import tune
    rods = inputs.uneven_rods(n_rods=4096, seed=0)
    Ns = np.array([r.N for r in rods])
    Ks = np.array([r.K for r in rods])
    k1 = tune.size_classes(Ns, Ks)
    rods2 = inputs.uneven_rods(n_rods=4096, seed=1)
    k2 = tune.size_classes(np.array([r.N for r in rods2]), np.array([r.K for r in rods2]))
    assert k1 == k2  # same distribution, same key
    k3 = tune.size_classes(Ns // 8 + 3, Ks)
    assert k3 != k1
    monkeypatch.setenv("HEAT1D_TUNE_CACHE", str(tmp_path / "c.json"))
    tune._store_cache("x", {"opts": {"elems_per_thread": 8}})
    assert tune._load_cache()["x"]["opts"]["elems_per_thread"] == 8


def test_candidates_are_valid_shapes():
    from paper_1510_08982_gb300 import tune
    for dt in ("float32", "float64"):
        for c in tune.batched_candidates(dt) + tune.stream_candidates(dt):
            assert c["elems_per_thread"] in (4, 8, 16) and c["block_threads"] % 32 == 0 and c["halo_steps"] >= 1


@pytest.mark.gpu
def test_tuned_batch_is_bit_identical(monkeypatch, tmp_path):
    import torch
    from paper_1510_08982_gb300 import build, heat1d, tune
    build.build()
    monkeypatch.setenv("HEAT1D_TUNE_CACHE", str(tmp_path / "c.json"))
    rods = inputs.uneven_rods(n_rods=300, seed=3, K_hi=2000)
    off, total = heat1d.pack_offsets([r.N for r in rods])
    specs = [(int(o), r.N, r.K, r.r, r.c1, r.cN) for o, r in zip(off, rods)]
    opts = tune.tune_batched(specs, "float32", n_sample=64, k_cap=500, reps=1,
                             candidates=[dict(elems_per_thread=8, block_threads=128, halo_steps=16),
                                         dict(elems_per_thread=16, block_threads=256, halo_steps=32)])
    assert tune.tune_batched(specs, "float32") == opts  # served from the cache
    u0 = np.zeros(total)
    for o, r in zip(off, rods):
        u0[o:o + r.N] = r.u0
    a = torch.tensor(u0, dtype=torch.float32, device="cuda")
    b = a.clone()
    with heat1d.Batch(specs, dtype="float32", **opts) as bt:
        bt.run(a)
        bt.sync()
    with heat1d.Batch(specs, dtype="float32") as bt:
        bt.run(b)
        bt.sync()
    assert torch.equal(a, b)
