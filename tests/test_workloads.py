"""Seeded input generators: the counter-based generator and the initial fields."""
import math

import numpy as np

from paper_1803_11345_gb300 import workloads as W


def test_splitmix64_reference_values():
    """SplitMix64 seeded with 0 starts 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4 (published
    reference outputs of the algorithm)."""
    z = W.splitmix64(0, np.arange(2, dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4


def test_spinodal_range_and_counter_access():
    phi = W.spinodal(64, 32, seed=5)
    assert phi.shape == (32, 64)
    assert phi.min() >= -0.05 and phi.max() < 0.05
    assert abs(phi.mean()) < 0.005
    # element (y, x) is stream element y*nx + x, regenerable on its own
    u = W.uniform01(5, 64 * 32)
    assert phi[3, 7] == 0.05 * (2 * u[3 * 64 + 7] - 1)


def test_droplet_and_layers():
    phi = W.droplet(64, 64, 16, gamma=0.04, a=0.04)
    assert phi[32, 32] > 0.99 and phi[0, 0] < -0.99
    lay = W.layers(4, 40, 10, 30, 0.04, 0.04)
    assert lay.shape == (40, 4) and lay[20, 0] > 0.99 and lay[0, 0] < -0.99
    assert math.isclose(W.interface_width(0.02, 0.04), 1.0)


def test_batch_members_ranges():
    mem = W.batch_members(256, seed=3)
    assert len(mem) == 256
    for m in mem:
        assert m["nx"] in (64, 128, 256, 512) and m["ny"] in (m["nx"], m["nx"] // 2)
        assert 1 <= m["zeta"] <= 1000 and 0.01 <= m["Ca"] <= 0.5
    kinds = {m["kind"] for m in mem}
    assert kinds == {"droplet", "spinodal"}
