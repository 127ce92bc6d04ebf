"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every test here checks the oracle (the CPU statement of arXiv:1803.00737
Sec. 2) against something other than itself: hand-worked fixtures, textbook
matrix forms, closed forms, invariants and brute force.  No GPU.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import matrices as M
from tests.conftest import read_golden

RNG = np.random.default_rng(12345)


# ------------------------------------------------------------------ P1: coefficients (Eq. 7-10)

def test_d4_coefficient_identities():
    h, g = O.d4_h(), O.d4_g()
    assert abs(h.sum() - math.sqrt(2)) < 1e-15
    assert abs((h * h).sum() - 1) < 1e-15
    assert abs(g.sum()) < 1e-15
    assert abs((g * g).sum() - 1) < 1e-15
    assert abs(h @ g) < 1e-15
    assert abs(h[0] * h[2] + h[1] * h[3]) < 1e-15  # double-shift orthogonality
    # two vanishing moments of the detail filter
    assert abs((np.arange(4) * g).sum()) < 1e-14


def test_d4_h_matches_textbook_closed_form():
    th, tg = M.d4_filters()
    np.testing.assert_allclose(O.d4_h(), th, rtol=0, atol=1e-16)
    np.testing.assert_allclose(O.d4_g(), tg, rtol=0, atol=1e-16)


def test_printed_g_fails_perfect_reconstruction():
    """Reading of Eq. 9-10: with g as printed, the literal Eq. 3-6 / 13-16 do not
    invert each other (and sum g != 0), so the oracle uses the quadrature mirror."""
    gp = O.d4_g_printed()
    assert abs(gp.sum()) > 0.1
    x = RNG.standard_normal(8)
    err = np.abs(O.idwt1d(O.dwt1d(x, 1, g=gp), 1, g=gp) - x).max()
    assert err > 0.1
    err_ok = np.abs(O.idwt1d(O.dwt1d(x, 1), 1) - x).max()
    assert err_ok < 1e-13


# ------------------------------------------------------------------ golden fixtures

def test_golden_haar_4x4_worked_example():
    gd = read_golden("haar_4x4_worked.txt")
    pan, ms = gd["pan"], gd["ms"]
    rows = np.stack([O.dwt1d(r, O.HAAR) for r in pan])
    np.testing.assert_array_equal(rows, gd["rows"])
    np.testing.assert_array_equal(O.dwt2(pan, O.HAAR), gd["dwt2"])
    fused = O.fuse(pan, [ms], O.HAAR)[0]
    np.testing.assert_array_equal(fused, gd["fused"])
    np.testing.assert_array_equal(O.to_u8(fused), gd["fused_u8"].astype(np.uint8))
    # the column-inverse stage, through the inverse of the swapped coefficients
    sw = gd["dwt2"].copy()
    sw[:2, :2] = ms
    cols = np.stack([O.idwt1d(c, O.HAAR) for c in sw.T]).T
    np.testing.assert_array_equal(cols, gd["cols_inv"])


def test_golden_d4_ramp():
    gd = read_golden("d4_ramp4_worked.txt")
    np.testing.assert_allclose(O.dwt1d(gd["s"][0], O.D4), gd["coeffs"][0], rtol=0, atol=1e-15)


# ------------------------------------------------------------------ P2: perfect reconstruction

@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("N", [2, 4, 6, 8, 10, 12, 14, 16])
def test_pr_1d(wav, N):
    x = RNG.integers(0, 256, N).astype(float)
    y = O.idwt1d(O.dwt1d(x, wav), wav)
    if wav == O.HAAR:
        np.testing.assert_array_equal(y, x)
    else:
        assert np.abs(y - x).max() < 1e-12


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("shape", [(2, 2), (4, 4), (4, 6), (8, 12), (6, 16), (64, 64), (34, 18)])
def test_pr_2d(wav, shape):
    if wav == O.D4 and min(shape) < 4:
        pytest.skip("D4 needs N >= 4 in the library; N = 2 covered in 1D")
    x = RNG.integers(0, 256, shape).astype(float)
    y = O.idwt2(O.dwt2(x, wav), wav)
    if wav == O.HAAR:
        np.testing.assert_array_equal(y, x)
    else:
        assert np.abs(y - x).max() < 1e-12


# ------------------------------------------------------------------ P3: brute-force matrices

def _matrix(fn, N):
    return np.stack([fn(e) for e in np.eye(N)], axis=1)


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("N", [2, 4, 6, 8, 12, 16])
def test_unit_vector_matrices_match_textbook(wav, N):
    A = _matrix(lambda e: O.dwt1d(e, wav), N)
    S = _matrix(lambda e: O.idwt1d(e, wav), N)
    At = M.analysis_matrix(N, wav)
    assert np.abs(A - At).max() < 1e-15
    if wav == O.D4:
        assert np.abs(S - A.T).max() < 1e-15          # literal Eq. 13-16 == transpose of Eq. 3-6
        assert np.abs(A @ A.T - np.eye(N)).max() < 1e-14
    else:
        assert np.abs(S - 2 * A.T).max() == 0.0       # /2 Haar: inverse is 2 A^T, not A^T
        assert np.abs(S @ A - np.eye(N)).max() == 0.0


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
def test_2d_is_kronecker_of_1d(wav):
    H, W = 4, 6
    AH, AW = M.analysis_matrix(H, wav), M.analysis_matrix(W, wav)
    K = np.kron(AH, AW)  # row-major vec: vec(A_H X A_W^T) = (A_H kron A_W) vec(X)
    J = np.stack([O.dwt2(e.reshape(H, W), wav).ravel() for e in np.eye(H * W)], axis=1)
    assert np.abs(J - K).max() < 1e-15


# ------------------------------------------------------------------ P4-P7: fusion

SHAPES = [(4, 4), (8, 12), (16, 6), (12, 20), (32, 32)]


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("shape", SHAPES)
def test_fuse_matches_closed_form(wav, shape):
    H, W = shape
    pan = RNG.integers(0, 256, shape).astype(float)
    ms = RNG.integers(0, 256, (3, H // 2, W // 2)).astype(float)
    F = O.fuse(pan, ms, wav)
    for b in range(3):
        cf = M.fuse_closed_form(pan, ms[b], wav, O.default_gain(wav))
        if wav == O.HAAR:
            np.testing.assert_array_equal(F[b], cf)
        else:
            assert np.abs(F[b] - cf).max() < 1e-11


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
def test_fuse_with_own_ll_returns_pan(wav):
    H, W = 16, 24
    pan = RNG.integers(0, 256, (H, W)).astype(float)
    ll = O.dwt2(pan, wav)[: H // 2, : W // 2] / O.default_gain(wav)
    F = O.fuse(pan, [ll], wav)[0]
    if wav == O.HAAR:
        np.testing.assert_array_equal(F, pan)
    else:
        assert np.abs(F - pan).max() < 1e-12


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
def test_constant_images(wav):
    H, W = 8, 12
    F = O.fuse(np.full((H, W), 7.0), [np.full((H // 2, W // 2), 7.0)], wav)[0]
    assert np.abs(F - 7.0).max() < 1e-12
    F = O.fuse(np.full((H, W), 7.0), [np.full((H // 2, W // 2), 100.0)], wav)[0]
    assert np.abs(F - 100.0).max() < 1e-12
    if wav == O.D4:  # reading R3: the D4 approximation of a constant c is 2c
        assert abs(O.dwt2(np.full((H, W), 7.0), wav)[0, 0] - 14.0) < 1e-12


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
def test_linearity(wav):
    H, W = 8, 10
    p1, p2 = RNG.standard_normal((2, H, W))
    m1, m2 = RNG.standard_normal((2, 2, H // 2, W // 2))
    a, b = 1.7, -0.3
    lhs = O.fuse(a * p1 + b * p2, a * m1 + b * m2, wav)
    rhs = a * O.fuse(p1, m1, wav) + b * O.fuse(p2, m2, wav)
    assert np.abs(lhs - rhs).max() < 1e-12


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
def test_point_evaluator_matches_whole_image(wav):
    H, W = 10, 14
    pan = RNG.integers(0, 256, (H, W)).astype(np.uint8)
    ms = RNG.integers(0, 256, (H // 2, W // 2)).astype(np.uint8)
    F = O.fuse(pan, [ms], wav)[0]
    ys, xs = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    pts = O.fuse_points(pan, ms, wav, ys.ravel(), xs.ravel())
    np.testing.assert_array_equal(pts, F.ravel())
    # the same from float inputs (the evaluator's other input path)
    pf, mf = RNG.uniform(0, 255, (H, W)), RNG.uniform(0, 255, (H // 2, W // 2))
    np.testing.assert_allclose(O.fuse_points(pf, mf, wav, ys.ravel(), xs.ravel()),
                               O.fuse(pf, [mf], wav)[0].ravel(), rtol=0, atol=1e-10)


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
def test_dwt2_point_evaluator_matches_whole_image(wav):
    H, W = 12, 10
    img = RNG.integers(0, 256, (H, W)).astype(np.uint8)
    Z = O.dwt2(img.astype(float), wav)
    ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    np.testing.assert_array_equal(O.dwt2_points(img, wav, ii.ravel(), jj.ravel()), Z.ravel())


# ------------------------------------------------------------------ P8: adjoint

ADJ_SHAPES = [(4, 4), (4, 6), (6, 4), (10, 14), (12, 8), (16, 20)]


def _all_points(H, W):
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    ii, jj = np.meshgrid(np.arange(H // 2), np.arange(W // 2), indexing="ij")
    return yy.ravel(), xx.ravel(), ii.ravel(), jj.ravel()


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
@pytest.mark.parametrize("shape", ADJ_SHAPES)
def test_adjoint_point_evaluator_matches_whole_image(wav, shape):
    """The lazy point-wise adjoint at every pixel equals the whole-image
    adjoint (itself pinned to the closed form, the explicit Jacobian and
    finite differences below).  Haar on integer gradients is exact."""
    H, W = shape
    B = 3
    G = RNG.integers(-50, 51, (B, H, W)).astype(float) if wav == O.HAAR else RNG.standard_normal((B, H, W))
    gp, gm = O.fuse_adjoint(G, wav)
    pp, pm = O.fuse_adjoint_points(G, wav, H, W, *_all_points(H, W))
    if wav == O.HAAR:
        np.testing.assert_array_equal(pp, gp.ravel())
        np.testing.assert_array_equal(pm, gm.reshape(B, -1))
    else:
        assert np.abs(pp - gp.ravel()).max() < 1e-13
        assert np.abs(pm - gm.reshape(B, -1)).max() < 1e-13


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
def test_adjoint_point_evaluator_matches_closed_form(wav):
    """P8 closed form: grad_MS_b = gain sigma^2 L_H G_b L_W^T and
    grad_PAN = sum_b (G_b - sigma^2 L_H^T L_H G_b L_W^T L_W), at every pixel."""
    H, W, B = 12, 10, 2
    G = RNG.standard_normal((B, H, W))
    gain = O.default_gain(wav)
    pp, pm = O.fuse_adjoint_points(G, wav, H, W, *_all_points(H, W))
    cgp = sum(M.adjoint_closed_form(G[b], wav, gain)[0] for b in range(B))
    cgm = np.stack([M.adjoint_closed_form(G[b], wav, gain)[1] for b in range(B)])
    assert np.abs(pp - cgp.ravel()).max() < 1e-12
    assert np.abs(pm - cgm.reshape(B, -1)).max() < 1e-12


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
def test_adjoint_point_evaluator_on_a_periodic_window(wav):
    """Given only a window of the output gradient that wraps past the image's
    last row and column, the points inside it (with a 4-pixel margin) equal the
    whole-image adjoint; a point whose taps leave the window is refused."""
    H, W, B = 16, 20, 2
    G = RNG.standard_normal((B, H, W))
    gp, gm = O.fuse_adjoint(G, wav)
    gy0, gx0, hg, wg = H - 5, W - 6, 12, 14          # rows 11..15, 0..6; columns 14..19, 0..7
    rows = (gy0 + np.arange(hg)) % H
    cols = (gx0 + np.arange(wg)) % W
    win = G[:, rows][:, :, cols]
    ys = np.array([14, 15, 0, 1, 2, 15, 0])
    xs = np.array([18, 19, 0, 1, 2, 0, 19])
    iis, jjs = np.array([7, 0, 0, 7]), np.array([9, 0, 9, 0])
    pp, pm = O.fuse_adjoint_points(win, wav, H, W, ys, xs, iis, jjs, gy0=gy0, gx0=gx0)
    assert np.abs(pp - gp[ys, xs]).max() < 1e-13
    assert np.abs(pm - gm[:, iis, jjs]).max() < 1e-13
    with pytest.raises(ValueError):
        O.fuse_adjoint_points(win, wav, H, W, [8], [4], gy0=gy0, gx0=gx0)


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
def test_adjoint_closed_form_and_dot_product(wav):
    H, W, B = 12, 16, 3
    G = RNG.standard_normal((B, H, W))
    gp, gm = O.fuse_adjoint(G, wav)
    gain = O.default_gain(wav)
    cgp = sum(M.adjoint_closed_form(G[b], wav, gain)[0] for b in range(B))
    cgm = np.stack([M.adjoint_closed_form(G[b], wav, gain)[1] for b in range(B)])
    assert np.abs(gp - cgp).max() < 1e-12
    assert np.abs(gm - cgm).max() < 1e-12
    if wav == O.HAAR:  # blocksum, not blockmean: the adjoint is not the inverse
        bs = G.reshape(B, H // 2, 2, W // 2, 2).sum(axis=(2, 4))
        assert np.abs(gm - bs).max() < 1e-12
    pan = RNG.standard_normal((H, W))
    ms = RNG.standard_normal((B, H // 2, W // 2))
    lhs = (O.fuse(pan, ms, wav) * G).sum()
    rhs = (pan * gp).sum() + (ms * gm).sum()
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
def test_adjoint_matches_explicit_matrices_64(wav):
    """The full Jacobian of the 64 x 64 one-band fusion, built column by column
    from the forward oracle, transposed, equals the backward oracle's matrix."""
    H = W = 64
    n, m = H * W, (H // 2) * (W // 2)
    zero_p, zero_m = np.zeros((H, W)), np.zeros((1, H // 2, W // 2))
    J = np.empty((n, n + m))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        J[:, k] = O.fuse(e.reshape(H, W), zero_m, wav)[0].ravel()
    for k in range(m):
        e = np.zeros(m)
        e[k] = 1.0
        J[:, n + k] = O.fuse(zero_p, e.reshape(1, H // 2, W // 2), wav)[0].ravel()
    K = np.empty((n + m, n))
    for k in range(n):
        e = np.zeros((1, n))
        e[0, k] = 1.0
        gp, gm = O.fuse_adjoint(e.reshape(1, H, W), wav)
        K[:, k] = np.concatenate([gp.ravel(), gm.ravel()])
    assert np.abs(K - J.T).max() < 1e-13


@pytest.mark.parametrize("wav", [O.HAAR, O.D4])
def test_adjoint_central_finite_differences_64(wav):
    """Central FD in FP64 of L = <G, fuse(P, M)> on a 64 x 64 scene, 2 bands."""
    H = W = 64
    B = 2
    pan = RNG.integers(0, 256, (H, W)).astype(float)
    ms = RNG.integers(0, 256, (B, H // 2, W // 2)).astype(float)
    G = RNG.standard_normal((B, H, W))
    gp, gm = O.fuse_adjoint(G, wav)
    idx = RNG.choice(H * W, 64, replace=False)
    for k in idx:
        d = np.zeros(H * W)
        d[k] = 1.0
        d = d.reshape(H, W)
        fd = ((O.fuse(pan + d, ms, wav) - O.fuse(pan - d, ms, wav)) * G).sum() / 2.0
        assert abs(fd - gp.ravel()[k]) < 1e-9
    for k in RNG.choice(B * (H // 2) * (W // 2), 64, replace=False):
        d = np.zeros(B * (H // 2) * (W // 2))
        d[k] = 1.0
        d = d.reshape(B, H // 2, W // 2)
        fd = ((O.fuse(pan, ms + d, wav) - O.fuse(pan, ms - d, wav)) * G).sum() / 2.0
        assert abs(fd - gm.ravel()[k]) < 1e-9


# ------------------------------------------------------------------ uint8 rule

def test_u8_clamp_and_round_half_even():
    x = np.array([-3.0, 0.4, 0.5, 1.5, 2.5, 3.5, 254.5, 255.4, 300.0, 127.49999, 127.5])
    np.testing.assert_array_equal(O.to_u8(x), [0, 0, 0, 2, 2, 4, 254, 255, 255, 127, 128])


# ------------------------------------------------------------------ P9: metrics

def test_q_index_identities():
    x = RNG.uniform(0, 255, (64, 96))
    y = RNG.uniform(0, 255, (64, 96))
    assert abs(O.q_index(x, x) - 1.0) < 1e-14
    assert abs(O.q_index(x, y) - O.q_index(y, x)) < 1e-15
    # ragged edge dropped: a 70 x 100 image gives the same Q as its 64 x 96 crop
    x2 = np.pad(x, ((0, 6), (0, 4)), constant_values=3.0)
    y2 = np.pad(y, ((0, 6), (0, 4)), constant_values=200.0)
    assert abs(O.q_index(x2, y2) - O.q_index(x, y)) < 1e-15


def test_q_index_affine_closed_form():
    """For y = a x + b on one window: Q = [2a/(1+a^2)] [2 mx (a mx + b) / (mx^2 + (a mx + b)^2)]."""
    x = RNG.uniform(10, 200, (32, 32))
    for a, b in [(1.0, 0.0), (0.5, 3.0), (2.0, -7.0), (-1.0, 300.0)]:
        mx = x.mean()
        my = a * mx + b
        expect = (2 * a / (1 + a * a)) * (2 * mx * my / (mx * mx + my * my))
        assert abs(O.q_index(x, a * x + b) - expect) < 1e-12


def test_q_index_degenerate_windows():
    c = np.full((32, 32), 5.0)
    assert O.q_index(c, c) == 1.0
    assert O.q_index(c, np.full((32, 32), 6.0)) == 0.0
    assert math.isnan(O.q_index(np.ones((16, 40)), np.ones((16, 40))))


def test_ergas_zero_and_offset_closed_form():
    H, W, B = 64, 64, 3
    ms = RNG.uniform(20, 200, (B, H // 2, W // 2))
    rep = ms.repeat(2, axis=1).repeat(2, axis=2)
    assert O.ergas(rep, ms) == 0.0
    d = np.array([1.0, -2.0, 4.0])
    mu = ms.mean(axis=(1, 2))
    expect = 50.0 * math.sqrt(np.mean(d ** 2 / mu ** 2))
    assert abs(O.ergas(rep + d[:, None, None], ms) - expect) < 1e-12


def test_qnr_identical_bands_is_one():
    H = W = 64
    pan = RNG.uniform(0, 255, (H, W))
    pan_lo = pan.reshape(H // 2, 2, W // 2, 2).mean(axis=(1, 3))
    fused = np.stack([pan] * 3)
    q, dl, ds = O.qnr(fused, [pan_lo] * 3, pan)
    assert abs(dl) < 1e-14 and abs(ds) < 1e-14 and abs(q - 1.0) < 1e-14


def test_qnr_single_band_has_no_spectral_distortion():
    H = W = 64
    pan = RNG.uniform(0, 255, (H, W))
    ms = RNG.uniform(0, 255, (1, H // 2, W // 2))
    fused = RNG.uniform(0, 255, (1, H, W))
    q, dl, ds = O.qnr(fused, ms, pan)
    assert dl == 0.0
    assert abs(q - (1.0 - ds)) < 1e-15


def test_qnr_spatial_term_closed_form():
    """F_l = a_l P + b_l and MS_l = PAN~: each Q(F_l, P) is the affine closed form
    per window and Q(MS_l, PAN~) = 1, so D_s = mean_l |1 - mean_w Qaff(w)|."""
    H = W = 64
    pan = RNG.uniform(10, 250, (H, W))
    pan_lo = pan.reshape(H // 2, 2, W // 2, 2).mean(axis=(1, 3))
    ab = [(1.0, 0.0), (0.8, 10.0)]
    fused = np.stack([a * pan + b for a, b in ab])
    _, _, ds = O.qnr(fused, [pan_lo, pan_lo], pan)
    terms = []
    for a, b in ab:
        qs = []
        for wy in range(2):
            for wx in range(2):
                mx = pan[32 * wy:32 * wy + 32, 32 * wx:32 * wx + 32].mean()
                my = a * mx + b
                qs.append((2 * a / (1 + a * a)) * (2 * mx * my / (mx * mx + my * my)))
        terms.append(abs(np.mean(qs) - 1.0))
    assert abs(ds - np.mean(terms)) < 1e-12


def test_qnr_spectral_term_and_product_closed_form():
    """Every band affine in one base image X: F_l = a_l X + b_l at PAN size,
    MS_l = c_l X~ + d_l at MS size (X~ the 2x2 block mean of X), PAN = X.  For
    y = p x + q and z = r x + s on a window of x with mean m, Q(y, z) =
    [2pr / (p^2 + r^2)] [2 mu_y mu_z / (mu_y^2 + mu_z^2)], mu = p m + q, r m + s;
    so D_lambda (mean over ordered pairs), D_s and QNR = (1 - D_lambda)(1 - D_s)
    all follow from the window means of X and X~, with both terms nonzero."""
    H = W = 128
    x = RNG.uniform(10, 250, (H, W))
    x_lo = x.reshape(H // 2, 2, W // 2, 2).mean(axis=(1, 3))
    fab = [(1.0, 0.0), (0.8, 10.0), (1.25, -5.0)]
    mcd = [(1.0, 2.0), (0.9, 0.0), (1.1, 4.0)]
    fused = np.stack([a * x + b for a, b in fab])
    ms = [c * x_lo + d for c, d in mcd]
    q, dl, ds = O.qnr(fused, ms, x)

    def win_means(img):
        n = img.shape[0] // 32, img.shape[1] // 32
        return [img[32 * i:32 * i + 32, 32 * j:32 * j + 32].mean() for i in range(n[0]) for j in range(n[1])]

    def q_aff(means, p, qq, r, s):
        out = []
        for m in means:
            mu_y, mu_z = p * m + qq, r * m + s
            out.append((2 * p * r / (p * p + r * r)) * (2 * mu_y * mu_z / (mu_y ** 2 + mu_z ** 2)))
        return np.mean(out)

    mh, ml = win_means(x), win_means(x_lo)
    B = len(fab)
    dl_ref = np.mean([abs(q_aff(mh, *fab[l], *fab[r]) - q_aff(ml, *mcd[l], *mcd[r]))
                      for l in range(B) for r in range(B) if l != r])
    ds_ref = np.mean([abs(q_aff(mh, *fab[l], 1.0, 0.0) - q_aff(ml, *mcd[l], 1.0, 0.0)) for l in range(B)])
    assert dl_ref > 1e-4 and ds_ref > 1e-4
    assert abs(dl - dl_ref) < 1e-12 and abs(ds - ds_ref) < 1e-12
    assert abs(q - (1.0 - dl_ref) * (1.0 - ds_ref)) < 1e-12
