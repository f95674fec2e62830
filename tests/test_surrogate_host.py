"""Host-side logic of the learned warm start: the start-up criteria on
synthetic Nusselt series and the roll-direction canonicalisation."""
import numpy as np
import pytest

from paper_2211_03160_gb300 import surrogate as S


def test_steps_to_steady_needs_the_band_held():
    nu = np.concatenate([np.ones(40), np.full(40, 5.0)])
    # trailing mean over 4 samples first equals 5 at sample 43 (window ends at 44)
    assert S.steps_to_steady(nu, 10, 4, 5.0, tol=0.01, hold=2) == 44 * 10
    # a series that only touches the band never holds
    spikes = np.tile([4.0, 6.0], 40)
    assert S.steps_to_steady(spikes, 1, 1, 5.0) is None


def test_steps_to_reach_is_the_first_passage():
    t = np.arange(200)
    rising = 5.0 * (1 - np.exp(-t / 20.0))
    k = S.steps_to_reach(rising, 3, 4, 5.0, tol=0.01)
    tm = np.convolve(rising, np.ones(4) / 4, mode="valid")
    first = int(np.argmax(np.abs(tm - 5.0) <= 0.05))
    assert k == (first + 4) * 3
    # a fluctuating, statistically steady series is reached at its first crossing
    osc = 5.0 + 2.0 * np.sin(t / 3.0 + 1.0)
    k = S.steps_to_reach(osc, 1, 1, 5.0)
    assert k is not None and k <= 12
    assert S.steps_to_steady(osc, 1, 1, 5.0) is None
    # a series that starts above the reference is reached when it first comes down to it
    above = 9.0 - 4.0 * (1 - np.exp(-t / 10.0))
    k = S.steps_to_reach(above, 1, 1, 5.0)
    assert np.all(above[:k - 1] > 5.05) and above[k - 1] <= 5.05


def test_canonical_roll_maps_mirror_images_together():
    n = 65
    yy, xx = np.meshgrid(np.linspace(0, 1, n), np.linspace(0, 1, n), indexing="ij")
    T = 0.5 - yy + 0.1 * np.sin(np.pi * xx) * np.sin(np.pi * yy) * (xx - 0.3)
    u = np.sin(np.pi * xx) * np.cos(np.pi * yy) * -1.0  # u < 0 on top: negative circulation
    v = -np.cos(np.pi * xx) * np.sin(np.pi * yy) * -1.0
    a = np.stack([T, u, v])[None]
    mirror = np.stack([T[:, ::-1], -u[:, ::-1], v[:, ::-1]])[None]
    ca, cm = S.canonical_roll(a), S.canonical_roll(mirror)
    assert np.array_equal(ca, cm)
    yc = (np.arange(n) - 0.5 * (n - 1))[:, None]
    assert (ca[0, 1] * yc).sum() > 0
    assert np.array_equal(S.canonical_roll(ca), ca)  # idempotent
    assert np.array_equal(a[0, 0], T)  # input untouched


def test_factor_rejects_unaligned_sizes():
    assert S.factor(513) == 8 and S.factor(129) == 2 and S.factor(65) == 1
    for bad in (64, 100, 514):
        with pytest.raises(ValueError):
            S.factor(bad)
