"""The serving request stream follows its stated recipe: Cu/W 50/50; bulk, vacancy, (001)
and (110) surfaces and indented snapshots uniformly; sizes log-uniform from 64 to 50,000
atoms (rounded to whole cells); 0-1000 K; a target ACE fraction uniform on [0, 1]; 1-100 MD
steps; Poisson arrivals at the given rate; the same stream for the same seed and count."""
import numpy as np

import synth


def test_serving_stream_recipe():
    n, rate = 300, 40.0
    reqs = synth.configs.serving_requests(n, seed=7, rate_per_s=rate)
    assert len(reqs) == n and [r["id"] for r in reqs] == list(range(n))
    species = np.array([r["species"] for r in reqs]) if "species" in reqs[0] else None
    if species is not None:
        cu = np.mean(species == "Cu")
        assert abs(cu - 0.5) < 4 * np.sqrt(0.25 / n)
    geoms = [r["geometry"] for r in reqs]
    counts = {g: geoms.count(g) for g in set(geoms)}
    assert set(counts) == set(synth.configs.GEOMETRIES) and len(counts) == 5
    for g, c in counts.items():
        assert abs(c / n - 0.2) < 4 * np.sqrt(0.16 / n), (g, c)
    atoms = np.array([len(r["x"]) for r in reqs])
    assert atoms.min() >= 32 and atoms.max() <= 70000
    # log-uniform on [64, 50000]: the median of log(size) sits at the midpoint, and each decade
    # holds its share (whole-cell rounding and removed atoms move sizes by tens of per cent)
    mid = 0.5 * (np.log(64) + np.log(50000))
    assert abs(np.median(np.log(atoms)) - mid) < 0.6
    assert np.mean(atoms < 1000) > 0.25 and np.mean(atoms > 5000) > 0.2
    steps = np.array([r["n_steps"] for r in reqs])
    assert steps.min() >= 1 and steps.max() <= 100 and abs(steps.mean() - 50.5) < 6.0
    T = np.array([r["temperature"] for r in reqs])
    f = np.array([r["ace_fraction_target"] for r in reqs])
    assert T.min() >= 0.0 and T.max() <= 1000.0 and f.min() >= 0.0 and f.max() <= 1.0
    assert abs(f.mean() - 0.5) < 0.07
    t = np.array([r["arrival_s"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0.0)
    assert abs(gaps.mean() * rate - 1.0) < 4.0 / np.sqrt(n)          # exponential gaps: sd = mean
    for r in reqs[:20]:
        assert r["x"].shape == (len(r["x"]), 3) and np.isfinite(r["x"]).all()
        assert r["v"].shape == r["x"].shape and r["region"]["kind"] == "sphere"
    # the same seed and count give the same stream (the arrival times are drawn first, for all
    # requests, so a shorter stream of the same seed is a different one)
    a1 = synth.configs.serving_requests(12, seed=11, rate_per_s=rate)
    a2 = synth.configs.serving_requests(12, seed=11, rate_per_s=rate)
    for a, b in zip(a1, a2):
        assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["v"], b["v"])
        assert a["n_steps"] == b["n_steps"] and a["arrival_s"] == b["arrival_s"] and a["region"] == b["region"]
