"""Host logic of the tensor-core synthesis: the pairing of azimuths phi and -phi (mod 2 pi) whose
table entries follow one from the other (Eqs. 7, 12: the cosine class is even and the sine class
odd in the azimuth difference). Checked on the CPU through vrte_azimuth_mirrors: every azimuth of
the grid is computed or stored from exactly one computed partner at minus its angle, and the
pairing finds every pair the grid holds."""
import math

import numpy as np
import pytest

import paper_1707_05882_gb300 as vr


def _check_pairing(phi):
    rep, mir = vr.azimuth_mirrors(phi)
    n = phi.size
    covered = np.concatenate([rep, mir[mir >= 0]])
    # each index once: computed, or stored from its partner
    assert np.array_equal(np.sort(covered), np.arange(n))
    assert np.all(np.diff(rep) > 0)
    for r, m in zip(rep, mir):
        if m >= 0:
            d = math.remainder(phi[r] + phi[m], 2 * math.pi)
            assert abs(d) <= 1e-12, (phi[r], phi[m])
            assert m != r
    # maximal: no two computed azimuths without partners are mirrors of each other
    lone = rep[mir < 0]
    for i in lone:
        for j in lone:
            if i < j:
                assert abs(math.remainder(phi[i] + phi[j], 2 * math.pi)) > 1e-12
    return rep, mir


@pytest.mark.parametrize("n", [1, 2, 7, 16, 90, 360])
def test_uniform_grid(n):
    phi = 2 * math.pi * np.arange(n) / n
    rep, mir = _check_pairing(phi)
    assert rep.size == n // 2 + 1          # 0 (and pi for even n) pair with themselves
    assert mir[0] == -1                    # phi = 0 is its own mirror


def test_irregular_grid_with_repeats_and_wrapped_angles():
    phi = np.array([0.3, 1.7, 4.0, 2 * math.pi - 0.3, math.pi, 0.0, 2 * math.pi - 1.7, 5.1,
                    1.7, -0.3, 7.0, 4 * math.pi - 7.0, 2.2])
    rep, mir = _check_pairing(phi)
    pairs = {(int(r), int(m)) for r, m in zip(rep, mir) if m >= 0}
    assert (0, 3) in pairs and (1, 6) in pairs and (10, 11) in pairs
    # the repeated 1.7 finds its only partner (-1.7) taken by the first one
    assert int(mir[list(rep).index(8)]) == -1


def test_grid_without_symmetry_computes_every_azimuth():
    rng = np.random.default_rng(7)
    phi = np.sort(rng.uniform(0.1, 3.0, 23))
    rep, mir = _check_pairing(phi)
    assert rep.size == 23 and np.all(mir == -1)


def test_invalid_arguments():
    lib = vr.load_library()
    assert lib.vrte_azimuth_mirrors(0, None, None, None) == 1
    with pytest.raises(vr.VrteError):
        vr.azimuth_mirrors(np.array([0.0, float("nan")]))
