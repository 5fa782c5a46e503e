"""The seeded input recipe: symmetric Cholesky vectors decaying like exp(-5P/n), pair-symmetric
amplitudes with sigma = 1e-2, float64 C-contiguous arrays, reproducible from the seed."""
import numpy as np

from paper_2310_04559_gb300 import synth


def test_cholesky_vectors_recipe():
    n, v = 400, 12
    L = synth.cholesky_vectors(n, v, seed=5)
    assert L.dtype == np.float64 and L.flags.c_contiguous and L.shape == (n, v, v)
    assert np.array_equal(L, L.transpose(0, 2, 1))  # L[P,a,c] = L[P,c,a]
    # undo the decay: the a <= c entries are standard normal, vector by vector
    X = L * np.exp(5.0 * np.arange(n) / n)[:, None, None]
    iu = np.triu_indices(v)
    x = X[:, iu[0], iu[1]]
    assert abs(x.mean()) < 0.02 and abs(x.std() - 1.0) < 0.02
    assert np.array_equal(L, synth.cholesky_vectors(n, v, seed=5))
    assert not np.array_equal(L, synth.cholesky_vectors(n, v, seed=6))
    G = synth.cholesky_vectors(n, v, seed=5, symmetric=False)
    assert not np.array_equal(G, G.transpose(0, 2, 1))


def test_amplitudes_recipe():
    o, v = 6, 30
    t = synth.amplitudes(o, v, seed=7)
    assert t.dtype == np.float64 and t.flags.c_contiguous and t.shape == (o, o, v, v)
    assert np.array_equal(t, t.transpose(1, 0, 3, 2))  # t_ijab = t_jiba
    # (X + X^swap)/2 of N(0, 1e-4) entries: off the i=j, a=b diagonal the std is 1e-2 / sqrt(2)
    i, j = np.triu_indices(o, 1)
    assert abs(t[i, j].std() - 1e-2 / np.sqrt(2)) < 3e-4
    assert np.array_equal(t, synth.amplitudes(o, v, seed=7))


def test_ladder_inputs_share_one_generator():
    L1, t1 = synth.ladder_inputs(3, 8, 20, seed=9)
    L2, t2 = synth.ladder_inputs(3, 8, 20, seed=9)
    assert np.array_equal(L1, L2) and np.array_equal(t1, t2)
    rng = np.random.default_rng(9)
    assert np.array_equal(L1, synth.cholesky_vectors(20, 8, rng=rng))
    assert np.array_equal(t1, synth.amplitudes(3, 8, rng=rng))
    Lov = synth.cholesky_ov(20, 3, 8, seed=1)
    assert Lov.shape == (20, 3, 8) and Lov.flags.c_contiguous
