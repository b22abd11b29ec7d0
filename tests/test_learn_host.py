"""Host side of the learned work estimator (no GPU): the parameter layout
include/mce.h documents, the rank correlation used to evaluate it, and the
committed model file the bench loads."""
import json
import os

import numpy as np
import pytest

from paper_2212_01473_gb300 import engine as E
from paper_2212_01473_gb300 import learn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
F, H = 16, 64


def test_parameter_count_matches_the_header_layout():
    # W1[64][16] b1[64] W2[64][64] b2[64] W3[64] b3 mean[16] std[16]
    assert E.MCE_MODEL_PARAMS == H * F + H + H * H + H + H + 1 + F + F


def test_init_params_layout():
    mean = np.arange(F, dtype=np.float64)
    std = np.linspace(0.0, 2.0, F)  # the first is floored at 1e-3
    p = learn.init_params(mean, std, seed=3)
    assert p.dtype == np.float32 and p.shape == (E.MCE_MODEL_PARAMS,)
    off = 0
    for fan_in, fan_out in ((F, H), (H, H), (H, 1)):
        w = p[off:off + fan_in * fan_out]
        lim = np.sqrt(6.0 / fan_in)
        assert np.all(np.abs(w) <= lim) and np.std(w) > 0.2 * lim  # He-uniform, not all zero
        off += fan_in * fan_out
        assert np.all(p[off:off + fan_out] == 0)  # biases start at zero
        off += fan_out
    assert off == E.MCE_MODEL_PARAMS - 2 * F
    assert np.array_equal(p[-2 * F:-F], mean.astype(np.float32))
    assert p[-F] == np.float32(1e-3) and np.array_equal(p[-F + 1:], std[1:].astype(np.float32))
    assert np.array_equal(learn.init_params(mean, std, seed=3), p)  # seeded


def test_spearman_matches_scipy():
    stats = pytest.importorskip("scipy.stats")
    rs = np.random.default_rng(1)
    a = rs.normal(size=500)
    b = a + rs.normal(scale=0.7, size=500)
    assert learn.spearman(a, b) == pytest.approx(stats.spearmanr(a, b)[0], abs=1e-12)
    assert learn.spearman(a, a) == pytest.approx(1.0)
    assert learn.spearman(a, -a) == pytest.approx(-1.0)


def test_committed_model_file():
    with open(os.path.join(ROOT, "paper_2212_01473_gb300", "work_model.json")) as f:
        d = json.load(f)
    p = np.array(d["params"], np.float64)
    assert p.shape == (E.MCE_MODEL_PARAMS,) and np.all(np.isfinite(p))
    assert np.all(p[-F:] > 0)  # every standard deviation is positive (mce_model_create requires it)
    assert "meta" in d
