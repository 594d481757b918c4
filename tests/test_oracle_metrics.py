"""Pins of the FP64 loss / metric reference on hand-computed inputs, and of
the oracle's fixed choices against the values the paper prints
(tests/golden/paper_hparams.json)."""
import json
import os

import numpy as np

import mg_synth as ms
from oracle import metrics, nrf

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_hparams.json")))


def test_l1_l2_hand_example():
    loss, g = metrics.l1_l2([1.0, 2.0, -1.0, 0.0], [0.0, 0.0, 0.0, 0.0])
    # mean |r| = 4/4 = 1, mean r^2 = 6/4 = 1.5
    assert abs(loss - 2.5) < 1e-15
    assert np.allclose(g, [(1 + 2) / 4, (1 + 4) / 4, (-1 - 2) / 4, 0.0])


def test_smooth_l1_eq_e11():
    v, g = metrics.smooth_l1([0.5, 2.0, -3.0, 0.0], [0.0, 0.0, 0.0, 0.0])
    # 0.5*0.25 = 0.125; 2 - 0.5 = 1.5; 3 - 0.5 = 2.5; 0
    assert abs(v - (0.125 + 1.5 + 2.5) / 4) < 1e-15
    assert np.allclose(g, [0.5 / 4, 1 / 4, -1 / 4, 0])


def test_psnr_and_aniso():
    a = np.zeros(100)
    b = np.full(100, 0.1)
    assert abs(metrics.psnr(a, b) - 20.0) < 1e-12
    assert abs(metrics.aniso(np.array([[1.0, 1.0, 3.0], [2.0, 2.0, 2.0]])) - 0.75) < 1e-15


def test_paper_constants():
    assert GOLD["params_per_gaussian"]["value"] == 3 + 4 + 3 + 1
    assert GOLD["nrf_fourier_bands"]["value"] == nrf.N_BANDS
    dims = ms.NRF_LAYERS["paper"]
    assert len(dims) - 1 == GOLD["nrf_hidden_layers"]["value"]
    assert all(o == GOLD["nrf_width"]["value"] for o, _ in dims[:-1])
    assert dims[0][1] == 3 + 6 * GOLD["nrf_fourier_bands"]["value"]
    assert nrf.NRFParams("paper", [], []).out_scale == GOLD["nrf_output_bound"]["value"]
