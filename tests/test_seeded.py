"""The shared seeded generator: SplitMix64 + Box-Muller, checked against the published definition."""
import numpy as np

from paper_2210_08816_gb300 import seeded

M = (1 << 64) - 1


def _splitmix_reference(state, n):
    out = []
    for _ in range(n):
        state = (state + 0x9E3779B97F4A7C15) & M
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        out.append(z ^ (z >> 31))
    return out


def test_splitmix_published_vector():
    # Outputs of SplitMix64 started from state 1234567 (Vigna's reference test vector).
    assert _splitmix_reference(1234567, 5) == [6457827717110365317, 3203168211198807973,
                                              9817491932198370423, 4593380528125082431,
                                              16408922859458223821]


def test_uniform_matches_scalar_definition():
    base = int(seeded._stream_base(7, 3))
    ref = _splitmix_reference(base, 16)
    u = seeded.uniform(7, 3, 16)
    expect = [((z >> 11) + 0.5) / 2.0 ** 53 for z in ref]
    assert np.array_equal(u, np.array(expect))


def test_normal_statistics_and_determinism():
    z = seeded.normal(0, 0, 400_000)
    assert abs(z.mean()) < 5e-3 and abs(z.std() - 1.0) < 5e-3
    assert np.array_equal(z[:1000], seeded.normal(0, 0, 1000))
    assert not np.array_equal(seeded.normal(0, 1, 1000), seeded.normal(0, 0, 1000))
    f = seeded.normal_fields(3, (4, 5, 6), sigma=2.0)
    assert len(f) == 4 and f[0].shape == (4, 5, 6)
