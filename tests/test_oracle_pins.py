"""Pins for the FP64 CPU oracle (no GPU).

Each test checks the oracle against something other than itself: a direct O(N^2)/O(N^4)
DFT, numpy/LAPACK routines the oracle does not use, the closed forms of Eq. 1 for a
point source and for the quadratic Gauss sum, the invariants of Eqs. 4-7 (Parseval,
C = I^T I, trace, PSD, SVD identity of Eqs. 2-3 and 5), and closed-form spectra.
Where useful, a test also shows that a plausible mistake (wrong DFT sign, wrong
retained range) would be caught.
"""

import numpy as np
import pytest

import oracle
from dh_synth import known_rank_frames, speckle_window

LAM, Z, PITCH = 785e-9, 0.35, 20e-6  # the workload's Fresnel parameters


def direct_dft1(x, sign):
    n = len(x)
    k = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / n) @ x


def direct_dft2(x, sign):
    ny, nx = x.shape
    ky, kx = np.arange(ny), np.arange(nx)
    Ey = np.exp(sign * 2j * np.pi * np.outer(ky, ky) / ny)
    Ex = np.exp(sign * 2j * np.pi * np.outer(kx, kx) / nx)
    # X[y, x] = sum_{l, k} x[l, k] Ey[y, l] Ex[x, k]  (written as an explicit 4-index sum)
    return np.einsum("yl,xk,lk->yx", Ey, Ex, x)


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


# ----------------------------------------------------------------------------- FFT
@pytest.mark.parametrize("n", [2, 4, 8, 16, 32])
@pytest.mark.parametrize("sign", [+1, -1])
def test_fft1d_matches_direct_dft(n, sign):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert rel(oracle.fft1d(x, sign), direct_dft1(x, sign)) < 1e-13


@pytest.mark.parametrize("shape", [(16, 16), (4, 8), (8, 4), (2, 16)])
def test_fft2d_matches_direct_dft(shape):
    rng = np.random.default_rng(7)
    xc = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    xr = rng.integers(0, 4096, size=shape).astype(np.float64)
    for x in (xc, xr):
        assert rel(oracle.fft2d(x, +1), direct_dft2(x, +1)) < 1e-13


def test_fft2d_matches_numpy_ifft2():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((64, 128)) + 1j * rng.standard_normal((64, 128))
    # numpy's ifft2 is (1/N) sum x exp(+2 pi i ...): the same kernel as Eq. 1's DFT.
    assert rel(oracle.fft2d(x, +1), np.fft.ifft2(x) * x.size) < 1e-13


def test_fft_sign_mistake_is_caught():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    assert rel(oracle.fft2d(x, -1), direct_dft2(x, +1)) > 0.5


# --------------------------------------------------------------------- Fresnel, Eq. 1
def fresnel_convolution_point(nx, ny, k0, l0, lam, z, pitch):
    """Eq. 1 as written (a convolution) for I = delta at pixel (k0, l0), sampled on the
    one-FFT output grid X = x lam z / (nx pitch), Y = y lam z / (ny pitch), without the
    constant prefactor."""
    x = np.arange(nx)[None, :] * lam * z / (nx * pitch)
    y = np.arange(ny)[:, None] * lam * z / (ny * pitch)
    xs = (k0 - nx // 2) * pitch  # centred source coordinates
    ys = (l0 - ny // 2) * pitch
    return np.exp(-1j * np.pi / (lam * z) * ((x - xs) ** 2 + (y - ys) ** 2))


@pytest.mark.parametrize("nx,ny", [(32, 16), (64, 64)])
def test_point_sources_match_fresnel_convolution(nx, ny):
    """Two point sources: the per-pixel ratio of their holograms is independent of the
    dropped output chirp, so it must equal the ratio of Eq. 1's convolution integrals."""
    sources = [(3, 5, 1000), (nx - 7, ny // 2 + 1, 250)]
    frames = np.zeros((2, ny, nx), dtype=np.uint16)
    for t, (k, l, A) in enumerate(sources):
        frames[t, l, k] = A
    H = oracle.render(frames, LAM, Z, PITCH)
    s = 1.0 / np.sqrt(nx * ny)
    for t, (k, l, A) in enumerate(sources):
        assert np.allclose(np.abs(H[t]), s * A, rtol=1e-12, atol=0)
    ratio = H[0] / H[1]
    (k0, l0, A0), (k1, l1, A1) = sources
    expect = (A0 / A1) * fresnel_convolution_point(nx, ny, k0, l0, LAM, Z, PITCH) / \
        fresnel_convolution_point(nx, ny, k1, l1, LAM, Z, PITCH)
    assert rel(ratio, expect) < 1e-10


def test_uniform_frame_quadratic_gauss_sum():
    """a = pitch^2/(lambda z) = 1/N makes each 1-D sum a quadratic Gauss sum of modulus
    sqrt(N): a uniform frame of value A gives |H| = s A N = A at every pixel."""
    N, A = 64, 1234
    z = PITCH ** 2 * N / LAM
    frames = np.full((1, N, N), A, dtype=np.uint16)
    H = oracle.render(frames, LAM, z, PITCH)
    assert np.allclose(np.abs(H[0]), A, rtol=1e-11)
    # a slightly different z breaks it (the pin sees the chirp coefficient)
    H2 = oracle.render(frames, LAM, z * 1.01, PITCH)
    assert np.max(np.abs(np.abs(H2[0]) - A)) > 1.0


def test_parseval_per_frame():
    f = speckle_window(32, 16, 4, seed=11).numpy()
    H = oracle.render(f, LAM, Z, PITCH)
    for t in range(4):
        e_raw = np.sum(f[t].astype(np.float64) ** 2)
        assert abs(np.sum(np.abs(H[t]) ** 2) - e_raw) <= 1e-12 * e_raw


# ------------------------------------------------------------------ covariance, Eq. 4
def test_covariance_equals_integer_gram_of_raw_frames():
    """Unitary chirp + unitary DFT preserve inner products per frame, so C = I^T I
    exactly; I^T I is computed here in int64 from the raw uint16 frames."""
    f = speckle_window(64, 32, 16, seed=2).numpy()
    H = oracle.render(f, LAM, Z, PITCH)
    C = oracle.covariance(H)
    I = f.reshape(16, -1).astype(np.int64)
    G = (I @ I.T).astype(np.float64)
    assert rel(C.real, G) < 1e-13
    assert np.max(np.abs(C.imag)) < 1e-13 * np.max(np.abs(G))


def test_covariance_hermitian_psd_trace():
    rng = np.random.default_rng(1)
    H = rng.standard_normal((8, 300)) + 1j * rng.standard_normal((8, 300))
    C = oracle.covariance(H)
    assert rel(C, C.conj().T) < 1e-15
    assert np.min(np.linalg.eigvalsh(C)) > -1e-12 * np.trace(C).real
    assert abs(np.trace(C).real - np.sum(np.abs(H) ** 2)) < 1e-12 * np.sum(np.abs(H) ** 2)
    # against numpy's matmul (BLAS), which the oracle does not use
    assert rel(C, H.conj() @ H.T) < 1e-13


# ----------------------------------------------------------------- eigen, Eq. 5
@pytest.mark.parametrize("T", [4, 16, 32, 64])
def test_eig_residual_orthonormal_and_lapack(T):
    rng = np.random.default_rng(T)
    X = rng.standard_normal((T, 3 * T)) + 1j * rng.standard_normal((T, 3 * T))
    C = X @ X.conj().T
    lam, V, sweeps = oracle.eig(C)
    nC = np.linalg.norm(C, 2)
    assert np.all(np.diff(lam) <= 0)
    assert np.linalg.norm(C @ V - V * lam[None, :]) <= 1e-12 * nC
    assert np.linalg.norm(V.conj().T @ V - np.eye(T)) <= 1e-13 * T
    assert abs(np.sum(lam) - np.trace(C).real) <= 1e-12 * nC * T
    ref = np.linalg.eigvalsh(C)[::-1]  # LAPACK heevd-type solver
    assert np.max(np.abs(lam - ref)) <= 1e-12 * nC
    assert sweeps <= 20


def test_eigenvalues_are_squared_singular_values():
    """Eq. 5 with Eq. 2: Lambda = Delta^2 for C = H^{t*} H."""
    f = speckle_window(32, 32, 8, seed=4).numpy()
    H = oracle.render(f, LAM, Z, PITCH).reshape(8, -1).T  # (n_x n_y, n_t)
    lam, _, _ = oracle.eig(oracle.covariance(H.T))
    sv = np.linalg.svd(H, compute_uv=False)
    assert np.max(np.abs(lam - sv ** 2)) <= 1e-12 * lam[0]


@pytest.mark.parametrize("T", [16, 32, 64])
def test_known_rank_spectrum(T):
    comps = [(1, 40, 300), (3, 25, 700), (T - 1, 10, 1500), (T // 2, 60, 90)]
    f, lam_exact = known_rank_frames(64, 64, T, 2000, comps, support_seed=T)
    H = oracle.render(f, LAM, Z, PITCH)
    lam, V, _ = oracle.eig(oracle.covariance(H))
    assert np.max(np.abs(lam - lam_exact)) <= 1e-11 * lam_exact[0]


def test_degenerate_and_diagonal_inputs():
    C = np.diag([5.0, 5.0, 1.0, 0.0]).astype(np.complex128)
    lam, V, sweeps = oracle.eig(C)
    assert np.allclose(lam, [5, 5, 1, 0]) and sweeps == 0
    assert np.allclose(np.abs(V), np.eye(4))


# -------------------------------------------------------------- projection, Eqs. 6-7
def _window(nx=32, ny=32, T=16, seed=9):
    f = speckle_window(nx, ny, T, seed=seed).numpy()
    return f, oracle.render(f, LAM, Z, PITCH)


def test_projection_parseval_full_range():
    f, H = _window()
    lam, V, _ = oracle.eig(oracle.covariance(H))
    M = oracle.project_power(H, V, 0, H.shape[0] - 1)
    assert rel(M, np.sum(np.abs(H) ** 2, axis=0)) < 1e-12


@pytest.mark.parametrize("k0,k1", [(2, 15), (0, 0), (5, 9), (15, 15)])
def test_projection_matches_svd_filter(k0, k1):
    """Eq. 3: H_f = U Delta I_f V^{t*}; sum_t |H_f|^2 equals M of Eqs. 6-7."""
    f, H = _window()
    T = H.shape[0]
    lam, V, _ = oracle.eig(oracle.covariance(H))
    M = oracle.project_power(H, V, k0, k1)
    Hs = H.reshape(T, -1).T
    U, sv, Vh = np.linalg.svd(Hs, full_matrices=False)  # decreasing singular values
    Hf = (U[:, k0:k1 + 1] * sv[k0:k1 + 1]) @ Vh[k0:k1 + 1, :]
    Mf = np.sum(np.abs(Hf) ** 2, axis=1).reshape(M.shape)
    assert rel(M, Mf) < 1e-10
    # an off-by-one retained range is a different image
    if k1 + 1 < T:
        assert rel(oracle.project_power(H, V, k0, k1 + 1), Mf) > 1e-3


def test_projection_diagonal_covariance():
    """Frames on disjoint pixel supports have a diagonal C: the components are the
    frames themselves (ordered by energy), so M is a sum of per-frame powers."""
    T, n = 8, 32
    f = np.zeros((T, n, n), dtype=np.uint16)
    rng = np.random.default_rng(0)
    perm = rng.permutation(n * n)
    energy = []
    for t in range(T):
        pix = perm[t * 40:(t + 1) * 40]
        vals = rng.integers(100, 4000, size=40) * (t + 1) // T + 1
        f[t].flat[pix] = vals
        energy.append(np.sum(vals.astype(np.float64) ** 2))
    H = oracle.render(f, LAM, Z, PITCH)
    lam, V, _ = oracle.eig(oracle.covariance(H))
    order = np.argsort(-np.array(energy), kind="stable")
    assert np.allclose(lam, np.array(energy)[order], rtol=1e-12)
    k0, k1 = 2, 6
    expect = np.sum(np.abs(H[order[k0:k1 + 1]]) ** 2, axis=0)
    assert rel(oracle.project_power(H, V, k0, k1), expect) < 1e-10


# ------------------------------------------------------------ whole window, numpy pipeline
def numpy_pipeline(frames, lam_m, z_m, pitch_m, k0, k1):
    """The same equations computed with numpy's FFT and LAPACK eigensolver."""
    T, ny, nx = frames.shape
    a = pitch_m ** 2 / (lam_m * z_m)
    kx, ky = np.arange(nx) - nx // 2, np.arange(ny) - ny // 2
    chirp2 = np.exp(-1j * np.pi * a * (ky[:, None] ** 2 + kx[None, :] ** 2))
    H = np.fft.ifft2(frames * chirp2, norm="ortho")
    Hs = H.reshape(T, -1).T
    C = Hs.conj().T @ Hs
    w, V = np.linalg.eigh(C)
    order = np.argsort(-w, kind="stable")
    w, V = w[order], V[:, order]
    P = Hs @ V[:, k0:k1 + 1]
    return np.sum(np.abs(P) ** 2, axis=1).reshape(ny, nx), w, C


@pytest.mark.parametrize("nx,ny,T", [(32, 16, 8), (64, 64, 16), (16, 16, 4)])
def test_pca_window_matches_numpy_pipeline(nx, ny, T):
    f = speckle_window(nx, ny, T, seed=nx + T).numpy()
    k0, k1 = 2, T - 1
    M, lam, C, _ = oracle.pca_window(f, LAM, Z, PITCH, k0, k1)
    Mn, wn, Cn = numpy_pipeline(f.astype(np.float64), LAM, Z, PITCH, k0, k1)
    assert rel(C, Cn) < 1e-12
    assert np.max(np.abs(lam - wn)) < 1e-12 * wn[0]
    assert rel(M, Mn) < 1e-9


def test_pca_window_rejects_bad_range():
    f = speckle_window(16, 16, 4, seed=1).numpy()
    with pytest.raises(RuntimeError):
        oracle.pca_window(f, LAM, Z, PITCH, 3, 4)


# ----------------------------------------------------------------- Eqs. 8-9 (Fourier)
def test_fourier_full_band_is_parseval():
    """W of Eq. 8 is unitary: keeping every bin returns sum_t |H_t|^2 per pixel."""
    rng = np.random.default_rng(5)
    H = rng.standard_normal((32, 8, 16)) + 1j * rng.standard_normal((32, 8, 16))
    M = oracle.fourier_power(H, 0, 31)
    assert np.allclose(M, (np.abs(H) ** 2).sum(0), rtol=1e-13, atol=0)


@pytest.mark.parametrize("T,k0,k1", [(32, 7, 23), (16, 3, 9), (64, 0, 5), (32, 31, 31)])
def test_fourier_matches_numpy_fft(T, k0, k1):
    """numpy's forward FFT with norm='ortho' is exactly Eq. 8's W (exp(-2 pi i t k / T) /
    sqrt(T)); the oracle writes the DFT out itself."""
    rng = np.random.default_rng(T + k0)
    H = rng.standard_normal((T, 4, 8)) + 1j * rng.standard_normal((T, 4, 8))
    F = np.fft.fft(H, axis=0, norm="ortho")
    ref = (np.abs(F[k0:k1 + 1]) ** 2).sum(0)
    assert np.allclose(oracle.fourier_power(H, k0, k1), ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("f", [3, 8, 29])
def test_fourier_complex_tone_lands_in_its_bin(f):
    """H_t = A exp(+2 pi i f t / T) is bin f of W exactly (|X_f|^2 = |A|^2 T, others 0):
    the sign of Eq. 8's exponent decides which bin, so a flipped sign (bin T - f) fails."""
    T = 32
    A = (1.5 - 0.5j) * np.ones((2, 2))
    t = np.arange(T)[:, None, None]
    H = A[None] * np.exp(2j * np.pi * f * t / T)
    assert np.allclose(oracle.fourier_power(H, f, f), np.abs(A) ** 2 * T, rtol=1e-12)
    others = [(0, f - 1)] if f > 0 else []
    others += [(f + 1, T - 1)] if f < T - 1 else []
    for a, b in others:
        assert np.max(oracle.fourier_power(H, a, b)) < 1e-20


def test_fourier_window_tone_closed_form():
    """Frames I_t = c0 + a cos(pi t / 2) on a pixel set: the Fresnel transform is linear and
    unitary per frame, so every pixel's temporal sequence is F(S)(p) (c0 + a cos(2 pi (T/4)
    t / T)), whose unitary DFT is c0 sqrt(T) at bin 0 and a sqrt(T) / 2 at bins T/4 and 3T/4.
    The paper's filter n_1 = 8, n_2 = 24 (bins 7..23 counted from 0) keeps bin 8 only, so
    M / sum_t |H_t|^2 = (a^2 T / 4) / (T c0^2 + a^2 T / 2) at every pixel; the bins 8..24
    (an off-by-one reading) would double it."""
    T, n, c0, a = 32, 16, 1000, 400
    rng = np.random.default_rng(9)
    S = rng.random((n, n)) < 0.3
    seq = c0 + a * np.round(np.cos(np.pi * np.arange(T) / 2)).astype(np.int64)
    frames = (seq[:, None, None] * S[None]).astype(np.uint16)
    M = oracle.fourier_window(frames, LAM, Z, PITCH, 7, 23)
    H = oracle.render(frames, LAM, Z, PITCH)
    P = (np.abs(H) ** 2).sum(0)
    mask = P > 1e-9 * P.max()
    ratio = (a * a * T / 4) / (T * c0 * c0 + a * a * T / 2)
    assert np.allclose(M[mask] / P[mask], ratio, rtol=1e-10)
    M2 = oracle.fourier_window(frames, LAM, Z, PITCH, 8, 24)
    assert np.allclose(M2[mask] / P[mask], 2 * ratio, rtol=1e-10)


# ------------------------------------------------- Eqs. 2-3 then 8-9 (SVD filter + DFT)
def test_svd_fourier_reduces_to_fourier_with_every_component():
    """I_f of Eq. 3 keeping every component leaves H_f = H (V unitary)."""
    f = speckle_window(16, 32, 16, seed=71).numpy()
    M, _ = oracle.svd_fourier_window(f, LAM, Z, PITCH, 0, 15, 3, 11)
    ref = oracle.fourier_window(f, LAM, Z, PITCH, 3, 11)
    assert np.allclose(M, ref, rtol=1e-9, atol=1e-12 * ref.max())


def test_svd_fourier_reduces_to_pca_with_every_bin():
    """Keeping every DFT bin, Eq. 9 is Parseval of H_f = (H V) I_f V^{t*}: the power of the
    kept principal components, i.e. the image of Eqs. 6-7."""
    f = speckle_window(32, 16, 32, seed=72).numpy()
    M, lam = oracle.svd_fourier_window(f, LAM, Z, PITCH, 2, 31, 0, 31)
    ref, lam_ref, _, _ = oracle.pca_window(f, LAM, Z, PITCH, 2, 31)
    assert np.allclose(M, ref, rtol=1e-9, atol=1e-12 * ref.max())
    assert np.allclose(lam, lam_ref, rtol=0, atol=1e-12 * lam_ref[0])


@pytest.mark.parametrize("k0,k1,b0,b1", [(2, 15, 3, 11), (5, 12, 0, 7), (0, 9, 8, 15)])
def test_svd_fourier_matches_numpy_svd_pipeline(k0, k1, b0, b1):
    """Eqs. 2-3 with numpy's SVD of the (pixels, n_t) matrix (singular values sorted
    decreasing, so index k of that order is kept for k0 <= k <= k1), then numpy's FFT."""
    f = speckle_window(16, 16, 16, seed=73 + k0).numpy()
    H = oracle.render(f, LAM, Z, PITCH).reshape(16, -1).T          # (pixels, n_t)
    U, d, Vh = np.linalg.svd(H, full_matrices=False)
    keep = np.zeros(16)
    keep[k0:k1 + 1] = 1.0
    Hf = (U * (d * keep)) @ Vh
    F = np.fft.fft(Hf, axis=1, norm="ortho")
    ref = (np.abs(F[:, b0:b1 + 1]) ** 2).sum(1).reshape(16, 16)
    M, lam = oracle.svd_fourier_window(f, LAM, Z, PITCH, k0, k1, b0, b1)
    assert np.allclose(M, ref, rtol=1e-8, atol=1e-10 * ref.max())
    assert np.allclose(lam, d ** 2, rtol=0, atol=1e-10 * d[0] ** 2)


# ------------------------------------------------------- display normalisation by the mean
def test_normalized_image_has_unit_mean_and_is_scale_free():
    rng = np.random.default_rng(80)
    M = rng.gamma(2.0, 3.0, size=(64, 32))
    N, mean = oracle.normalize(M)
    assert abs(N.mean() - 1.0) < 1e-14 and np.isclose(mean, M.sum() / M.size, rtol=1e-14)
    N2, _ = oracle.normalize(7.5 * M)
    assert np.allclose(N, N2, rtol=1e-14)


def test_display_codes_of_known_images():
    """A constant image shows the mean's code; 2x the mean and above saturate; 0 is black.
    The codes come from the image's own mean."""
    const = np.full((8, 8), 3.25)
    assert np.all(oracle.display_u8(const) == 128)
    # mean 16/6, so 128 / mean = 48 exactly: codes 48 M, saturating above 255
    ramp = np.array([0.0, 1.0, 2.0, 3.0, 4.0, 6.0])
    assert list(oracle.display_u8(ramp)) == [0, 48, 96, 144, 192, 255]
    # gain 64: mean -> 64, and a value at 1.5 x the mean sits exactly on 96
    img = np.array([1.0, 1.0, 1.0, 1.0, 1.5, 0.5])
    assert list(oracle.display_u8(img, 64.0)) == [64, 64, 64, 64, 96, 32]
    # round half to even, as rint does: 2.5 -> 2 at gain 2.5 / 1.0
    assert list(oracle.display_u8(np.array([1.0, 1.0]), 2.5)) == [2, 2]
