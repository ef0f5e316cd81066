"""The seeded workload builders: the CNN's convolution graph is the strided
valid convolution it stands for (pinned against scipy's 2-D correlation, an
implementation that shares nothing with the CSR builder)."""
import numpy as np
import pytest

from paper_2110_13638_gb300 import workloads as W

signal = pytest.importorskip("scipy.signal")


def _csr_apply(node, x):
    rp, ci, w = node["row_ptr"], node["col_idx"], node["weight"]
    return np.array([np.dot(w[rp[o]:rp[o + 1]], x[ci[rp[o]:rp[o + 1]]]) for o in range(len(rp) - 1)])


def _direct(K, img, stride):
    return np.concatenate([signal.correlate2d(img, K[f], mode="valid")[::stride, ::stride].reshape(-1)
                           for f in range(K.shape[0])])


def test_conv_csr_equals_strided_valid_correlation():
    rng = np.random.default_rng(5)
    for H, Wd, F, k, st in ((28, 28, 5, 5, 2), (7, 9, 2, 3, 1), (8, 6, 3, 2, 3)):
        K = rng.normal(size=(F, k, k))
        rp, ci, cv, n = W.conv_csr(K, H, Wd, st)
        node = {"row_ptr": rp, "col_idx": ci, "weight": cv}
        img = rng.uniform(size=(H, Wd))
        want = _direct(K, img, st)
        assert n == want.size
        assert np.allclose(_csr_apply(node, img.reshape(-1)), want, atol=1e-12)


def test_cnn_conv_node_is_conv5x5_stride2():
    g, x = W.cfg1()
    conv = g["nodes"][1]
    assert conv["kind"] == "linear" and conv["n_out"] == 720 and x.shape == (784, 8192)
    rp = conv["row_ptr"]
    assert np.all(np.diff(rp) == 25)
    # filters read off the first output of each filter map (row f * 144, columns dr * 28 + dc)
    K = np.zeros((5, 5, 5))
    for f in range(5):
        o = f * 144
        for c, w in zip(conv["col_idx"][rp[o]:rp[o + 1]], conv["weight"][rp[o]:rp[o + 1]]):
            K[f, c // 28, c % 28] = w
    assert np.all(K != 0)
    for j in (0, 17, 8191):
        img = x[:, j].reshape(28, 28)
        assert np.allclose(_csr_apply(conv, x[:, j]), _direct(K, img, 2), atol=1e-12)
    # He-normal, fan-in 25: std sqrt(2/25) = 0.283 (125 draws)
    assert 0.18 < np.std(K) < 0.39
