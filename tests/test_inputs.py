"""The seeded input generators both sides are fed from (CPU only).

SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) against a scalar restatement of its published
definition and the widely quoted first outputs for seed 0; the uniform and normal mappings;
the workload recipes' shapes and value ranges.
"""
import numpy as np

from paper_2502_08370_gb300 import workloads as wl

MASK = (1 << 64) - 1


def splitmix_scalar(seed, n):
    x, out = seed & MASK, []
    for _ in range(n):
        x = (x + 0x9E3779B97F4A7C15) & MASK
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_first_outputs_seed_0():
    got = [int(v) for v in wl.SplitMix64(0).next_u64(3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_splitmix64_matches_definition_across_calls():
    for seed in (1, 2, 12345, 2 ** 63 + 7):
        r = wl.SplitMix64(seed)
        got = [int(v) for v in r.next_u64(5)] + [int(v) for v in r.next_u64(1)] + [int(v) for v in r.next_u64(9)]
        assert got == splitmix_scalar(seed, 15), seed


def test_uniform_uses_the_top_53_bits_and_normals_are_standard():
    r = wl.SplitMix64(9)
    raw = splitmix_scalar(9, 4)
    u = r.uniform(4)
    assert np.array_equal(u, np.array([(v >> 11) / 2.0 ** 53 for v in raw]))
    z = wl.SplitMix64(10).normal(200000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01
    assert abs(np.mean(z ** 4) - 3.0) < 0.05  # Gaussian kurtosis
    k = wl.SplitMix64(11).integers(1, 63, 100000)
    assert k.min() == 1 and k.max() == 63 and abs(k.mean() - 32.0) < 0.2


def test_workload_recipes_shapes_and_ranges():
    c1 = wl.heat2d_63(n=15, N=4, s=8)
    assert c1["u0"].shape == (15, 15) and c1["a"] is None and c1["src"] is None
    c2 = wl.heat3d_255(n=9, N=4, s=4)
    assert c2["u0"].shape == (9, 9, 9) and c2["a"].shape == (11, 11, 11) and c2["src"].shape == (9, 9, 9)
    assert 0.5 - 1e-12 <= c2["a"].min() and c2["a"].max() <= 1.5 + 1e-12
    # the same seed gives the same inputs; another seed other ones
    assert np.array_equal(wl.heat2d_63(n=15, N=4, s=8)["u0"], c1["u0"])
    assert not np.array_equal(wl.heat2d_63(n=15, N=4, s=8, seed=7)["u0"], c1["u0"])


def test_full_tensor_coefficients_are_spd():
    d, b = wl.full_tensor_coefficients(31, 17)
    assert d.shape == b.shape == (19, 33)
    assert d.min() >= 1.0 / 3.0 - 1e-15 and d.max() <= 1.0 + 1e-15
    assert np.all(d * d - b * b >= 7.0 / 144.0 - 1e-15)  # d11 d22 - d12^2 >= 1/9 - 1/16
