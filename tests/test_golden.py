"""The oracle's conventions against what the paper fixes exactly (fixtures in tests/golden/).

The paper prints no worked numerical example; it does fix the DFT basis of Eq. 8 and the
filter indices of its two demodulations (text after Eq. 9). These tests read those from the
fixtures and check that the oracle's Fourier power and its PCA window follow them:
- a temporal tone along a column of Eq. 8's W lands in that column's bin only (a flipped
  sign would put it in bin n_t - j);
- the paper's PCA range, eigenvalues 1..20 of 32 in increasing order, is the oracle's
  range k0 = 12 .. k1 = 31 of the decreasing order, and its Fourier range n_1 = 8 .. n_2 = 24
  is the oracle's bins 7..23 (counted from 0).
"""

import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [line.split() for line in f if line.strip() and not line.startswith("#")]


def test_eq8_basis_matches_fixture_and_oracle_sign():
    rows = _rows("eq8_dft_basis_nt4.txt")
    n_t = 4
    W = np.zeros((n_t, n_t), dtype=np.complex128)
    for m, n, re, im in rows:
        W[int(m) - 1, int(n) - 1] = float(re) + 1j * float(im)
    # the fixture is Eq. 8 written out, and W is unitary
    m = np.arange(1, n_t + 1)[:, None]
    n = np.arange(1, n_t + 1)[None, :]
    assert np.allclose(W, np.exp(-2j * (m - 1) * (n - 1) * np.pi / n_t) / np.sqrt(n_t), atol=1e-15)
    assert np.allclose(W.conj().T @ W, np.eye(n_t), atol=1e-15)
    # H_t = conj(w_{t, j}) at every pixel: sum_t H_t w_{t, k} = delta_jk, so all the power is
    # in bin j (0-based j = n - 1) and none in the others
    for j in range(n_t):
        H = np.repeat(np.conj(W[:, j])[:, None, None], 2, axis=1).repeat(3, axis=2)
        for k in range(n_t):
            P = oracle.fourier_power(H, k, k)
            assert np.allclose(P, 1.0 if k == j else 0.0, atol=1e-12), (j, k, P.ravel()[0])


def test_filter_indices_map_to_oracle_ranges():
    rows = {r[0]: (int(r[1]), int(r[2]), int(r[3])) for r in _rows("filter_indices_nt32.txt")}
    n_t, n1, n2 = rows["pca"]
    rng = np.random.default_rng(7)
    # a small stack of holograms with distinct eigenvalues
    H = rng.standard_normal((n_t, 6, 5)) + 1j * rng.standard_normal((n_t, 6, 5))
    H *= np.linspace(1.0, 3.0, n_t)[:, None, None]
    Hm = H.reshape(n_t, -1)
    C = Hm.conj() @ Hm.T
    # the paper's form: eigenvalues increasing, keep eigenvectors n1..n2 (1-based), Eqs. 6-7
    lam, V = np.linalg.eigh(C)
    paper = (np.abs(Hm.T @ V[:, n1 - 1:n2]) ** 2).sum(axis=1)
    # the oracle's decreasing order: the same components are k0 = n_t - n2 .. k1 = n_t - n1
    k0, k1 = n_t - n2, n_t - n1
    assert (k0, k1) == (12, 31)
    ours = oracle.project_power(H, oracle.eig(C)[1], k0, k1).ravel()
    assert np.allclose(ours, paper, rtol=1e-9, atol=1e-9 * paper.max())
    # Fourier: the paper's n_1..n_2 = 8..24 are bins 7..23 counted from 0
    n_t, f1, f2 = rows["fourier"]
    assert (f1 - 1, f2 - 1) == (7, 23)
    tone = np.exp(2j * np.pi * np.arange(n_t) * 7 / n_t)[:, None, None] * np.ones((1, 2, 2))
    # a tone at bin 7 (0-based) is kept by bins [f1 - 1, f2 - 1] and lost by the symmetric
    # alternative [f1, f2]
    assert np.allclose(oracle.fourier_power(tone, f1 - 1, f2 - 1), n_t)
    assert np.allclose(oracle.fourier_power(tone, f1, f2), 0.0, atol=1e-9)
