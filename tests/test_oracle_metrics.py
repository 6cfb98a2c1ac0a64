"""Pins for the Sec. IV metrics against Table 2."""

import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import ising, metrics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_comparisons.json")


def test_tts_and_speed_reproduce_table2():
    g = json.load(open(GOLDEN))
    for name, row in g["rows"].items():
        tts = metrics.tts(row["T"], row["chi_hat"], g["d"])
        assert tts == pytest.approx(row["TTS"], rel=5e-3), name
        assert metrics.speed(row["T"], row["chi_hat"]) == pytest.approx(row["v"], rel=1.5e-2), name


def test_chi_hat_end_points():
    inst = synth.sk_dense(30, 1, 1.0, h_std=1.0)
    A, b = ising.paper_form(inst)
    emax = math.sqrt(30) * np.linalg.norm(A) + np.abs(b).sum()
    assert metrics.chi_hat(inst, -emax) == pytest.approx(1.0)
    assert metrics.chi_hat(inst, 0.0) == pytest.approx(0.5)
    assert metrics.chi_hat(inst, emax) == pytest.approx(0.0)


def test_pruning_rate():
    assert metrics.pruning_rate(1000, 51) == pytest.approx(0.949)
