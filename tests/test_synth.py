"""The seeded input generators: Philox4x32-10 known answers, the series
logarithm, Gaussian moments, SU(3) links, strong-coupling plaquette, and
bitwise reproducibility against checksums written on another machine."""
import json
import math
import os

import numpy as np
import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def test_philox_known_answers():
    # Random123 known-answer vectors for Philox4x32-10
    assert [hex(x) for x in synth.philox4x32_10([0, 0, 0, 0], [0, 0])] == \
        ["0x6627e8d5", "0xe169c58d", "0xbc57ac4c", "0x9b00dbd8"]
    assert [hex(x) for x in synth.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2)] == \
        ["0x408f276d", "0x41c83b0e", "0xa20bc7c6", "0x6d5451fd"]
    assert [hex(x) for x in synth.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
                                                [0xA4093822, 0x299F31D0])] == \
        ["0xd16cfe09", "0x94fdcceb", "0x5001e420", "0x24126ea1"]


@pytest.mark.parametrize("x", [1e-300, 1e-10, 0.3, 0.70710678, 1.0, 1.5, 2.0, 7.3e12])
def test_series_log(x):
    assert abs(synth.log(x) - math.log(x)) <= 4e-16 * max(1.0, abs(math.log(x)))


def test_gaussian_moments():
    g = synth.gaussian(400000, 11, 3)
    for part in (g.real, g.imag):
        assert abs(part.mean()) < 5e-3 and abs(part.var() - 1) < 1e-2
    assert abs((g.real * g.imag).mean()) < 5e-3


def test_links_are_su3():
    L = (4, 4, 2, 4)
    U = synth.gauge_field(L, beta=6.0, sweeps=3, n_or=1, seed=4, cache=False).reshape(-1, 3, 3)
    eye = np.eye(3)
    assert np.abs(U @ U.conj().transpose(0, 2, 1) - eye).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14


def test_strong_coupling_plaquette():
    """Leading strong-coupling behaviour <P> = beta/18 + O(beta^2) for SU(3)."""
    L = (4, 4, 4, 4)
    beta = 0.3
    U = synth.hot_gauge(L, 8)
    vals = []
    for s in range(40):
        synth.gauge_sweep(U, L, beta, 1, 8, s)
        if s >= 10:
            vals.append(synth.plaquette(U, L))
    p = float(np.mean(vals))
    assert abs(p - beta / 18 - beta ** 2 / 216) < 3e-3, p


def test_bitwise_reproducible_against_recorded_checksums():
    ref = json.load(open(os.path.join(HERE, "golden", "synth_checksums.json")))
    import tests.golden.make_synth_checksums as mk
    got = mk.compute()
    for k, v in ref.items():
        assert got[k]["sha1"] == v["sha1"], k
