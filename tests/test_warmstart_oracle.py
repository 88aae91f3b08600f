"""The FP64 reference of the warm-start network, pinned by finite
differences and hand-computed cases (CPU)."""
import numpy as np

from oracle import warmstart as ws


def random_params(n_out, seed):
    rng = np.random.default_rng(seed)
    parts = []
    for fi, fo in ws.shapes(n_out):
        parts += [rng.normal(0, 1.0 / np.sqrt(fi), fi * fo), rng.normal(0, 0.1, fo)]
    return np.concatenate(parts)


def test_gradients_match_finite_differences():
    n_out = 5
    p = random_params(n_out, 1)
    rng = np.random.default_rng(2)
    Y = rng.uniform(-1, 1, (2, 7, 3))
    tgt = rng.normal(0, 1, (2, n_out))
    g = ws.gradients(p, Y, tgt, n_out)
    idx = rng.choice(p.size, 60, replace=False)
    # include the first weights of every layer
    o = 0
    for fi, fo in ws.shapes(n_out):
        idx = np.append(idx, [o, o + fi * fo])
        o += fi * fo + fo
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (ws.loss(ws.forward(p + e, Y, n_out)[0], tgt) - ws.loss(ws.forward(p - e, Y, n_out)[0], tgt)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_forward_on_a_hand_case():
    # one point, identity-like layers: the network reduces to a chain of ReLUs
    n_out = 2
    P = []
    for fi, fo in ws.shapes(n_out):
        W = np.zeros((fi, fo))
        for k in range(min(fi, fo)):
            W[k, k] = 1.0
        P += [W.ravel(), np.zeros(fo)]
    p = np.concatenate(P)
    Y = np.array([[[0.5, -2.0, 3.0]]])
    pred, a = ws.forward(p, Y, n_out)
    np.testing.assert_allclose(pred, [[0.5, 0.0]])      # negative coordinate cut by the ReLUs
    # the max over points takes each feature's largest value
    Y2 = np.array([[[0.5, 1.0, 0.0], [0.25, 2.0, 1.0]]])
    pred2, a2 = ws.forward(p, Y2, n_out)
    np.testing.assert_allclose(a2["g"][0, :3], [0.5, 2.0, 1.0])
    np.testing.assert_allclose(pred2, [[0.5, 2.0]])


def test_permutation_invariance():
    n_out = 4
    p = random_params(n_out, 3)
    rng = np.random.default_rng(4)
    Y = rng.uniform(-1, 1, (1, 20, 3))
    perm = rng.permutation(20)
    np.testing.assert_allclose(ws.forward(p, Y, n_out)[0], ws.forward(p, Y[:, perm], n_out)[0], rtol=1e-14)
