"""Seeded input generators (workloads/): determinism and the relations
between generated columns. No GPU needed."""
import numpy as np

import workloads


def test_phase_space_snapshot_is_seeded_and_consistent():
    """The fused multi-grid workload's columns: the same seed gives the same
    snapshot, and the derived scalars follow from the base columns."""
    a = workloads.phase_space(5000, seed=3)
    b = workloads.phase_space(5000, seed=3)
    c = workloads.phase_space(5000, seed=4)
    assert list(a) == ["x", "y", "z", "vx", "vy", "vz", "mass", "speed", "ke", "r", "phi", "lz", "ly"]
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    assert not np.array_equal(a["x"], c["x"])
    v2 = a["vx"] ** 2 + a["vy"] ** 2 + a["vz"] ** 2
    np.testing.assert_allclose(a["speed"] ** 2, v2, rtol=1e-12)
    np.testing.assert_allclose(a["ke"], 0.5 * a["mass"] * v2, rtol=1e-12)
    np.testing.assert_allclose(a["lz"], a["x"] * a["vy"] - a["y"] * a["vx"], rtol=1e-12, atol=1e-12)
    assert (a["r"] < 10.0).all() and (a["mass"] >= 1.0).all() and (a["mass"] < 2.0).all()
    assert set(workloads.PHASE_SPACE_VARIABLES) <= set(a)
    for p, q in workloads.PHASE_SPACE_SYSTEMS:
        assert p in workloads.PHASE_SPACE_BOUNDS and q in workloads.PHASE_SPACE_BOUNDS
