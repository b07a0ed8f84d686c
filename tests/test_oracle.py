"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Every test compares the oracle with something other than itself: values worked out by
hand from Fig. 3's rule (tests/golden/), closed forms, library routines for special
cases, invariants of the method, and an independent naive restatement on tiny inputs.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import ndimage

from oracle import naive

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rng_img(rng, H, W):
    return rng.integers(0, 256, size=(H, W, 3), dtype=np.uint8)


# ----------------------------------------------------------------------------- depth map
def test_luma_grey_is_identity(oracle):
    v = np.arange(256, dtype=np.uint8)
    img = np.stack([v, v, v], axis=-1)[None]
    assert np.array_equal(oracle.luma(img)[0], v)


def test_luma_primaries_textbook(oracle):
    # BT.601 8-bit luma of the pure primaries: 0.299*255 = 76.245, 0.587*255 = 149.685,
    # 0.114*255 = 29.07  ->  76, 150, 29 (a transposed or wrong weight fails here)
    img = np.array([[[255, 0, 0], [0, 255, 0], [0, 0, 255], [255, 255, 255], [0, 0, 0]]], np.uint8)
    assert oracle.luma(img)[0].tolist() == [76, 150, 29, 255, 0]


def test_luma_exhaustive_against_fp64_with_tie_rule(oracle):
    # all 2^24 colours: FP64 evaluation of the BT.601 sum, where an exact half (the true
    # value has at most three decimals) is recognised explicitly and rounded up
    n = np.arange(1 << 24, dtype=np.uint32)
    img = np.stack([(n >> 16) & 255, (n >> 8) & 255, n & 255], axis=-1).astype(np.uint8)
    img = img.reshape(4096, 4096, 3)
    y = oracle.luma(img).reshape(-1).astype(np.int64)
    r, g, b = (img.reshape(-1, 3).astype(np.float64).T)
    v = 0.299 * r + 0.587 * g + 0.114 * b
    fl = np.floor(v)
    frac = v - fl
    expect = np.where(np.abs(frac - 0.5) < 1e-6, fl + 1, np.floor(v + 0.5)).astype(np.int64)
    assert np.array_equal(y, expect)


def test_binom5_matches_scipy_correlate(oracle):
    rng = np.random.default_rng(1)
    k = np.outer([1, 4, 6, 4, 1], [1, 4, 6, 4, 1]).astype(np.float64)
    for (H, W) in [(1, 1), (1, 7), (7, 1), (2, 3), (5, 5), (13, 31), (64, 48)]:
        Y = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
        S = ndimage.correlate(Y.astype(np.float64), k, mode="nearest")  # clamp-to-edge
        expect = np.floor(S / 256.0 + 0.5).astype(np.uint8)  # S/256 is exact in FP64
        assert np.array_equal(oracle.smooth_binom5(Y), expect), (H, W)


def test_binom5_constant_and_step(oracle):
    Y = np.full((9, 11), 173, np.uint8)
    assert np.array_equal(oracle.smooth_binom5(Y), Y)
    # a vertical step edge 0 | 255: rows identical, columns follow the 1-D binomial CDF
    Y = np.zeros((6, 10), np.uint8)
    Y[:, 5:] = 255
    D = oracle.smooth_binom5(Y)
    cdf = {3: 1, 4: 5, 5: 11, 6: 15}  # partial sums of [1 4 6 4 1] reaching the 255 side
    for x in range(10):
        s = 255 * (16 if x >= 7 else cdf.get(x, 0)) * 16
        assert (D[:, x] == (s + 128) // 256).all(), x


# ------------------------------------------------------------------------- shift tables
def _read_lut_golden():
    rows = []
    with open(os.path.join(GOLDEN, "lut_p16.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(tuple(int(v) for v in line.split()))
    return rows


def test_lut_golden_p16(oracle):
    hL, hR = oracle.disparity_lut(0, 16, 150)
    for d, l, r in _read_lut_golden():
        assert (hL[d], hR[d]) == (l, r), d


@pytest.mark.parametrize("P", [0, 1, 2, 3, 4, 5, 16, 63, 64, 65, 192, 511, 1024])
@pytest.mark.parametrize("T", [0, 150, 254, 255])
def test_lut_paper_rule_exact_rational(oracle, P, T):
    hL, hR = oracle.disparity_lut(0, P, T)
    for d in range(256):
        s = (-Fraction(P, 2) * Fraction(d, 255)) if d > T else Fraction(P, 2) * (1 - Fraction(d, 255))
        assert hL[d] == math.floor(s) and hR[d] == math.floor(-s), (P, T, d)


@pytest.mark.parametrize("P", [0, 1, 7, 16, 64, 1024])
def test_lut_invariants(oracle, P):
    for rule in (0, 1):
        hL, hR = oracle.disparity_lut(rule, P, 150)
        hL, hR = hL.astype(int), hR.astype(int)
        assert (np.diff(hL) <= 0).all() and (np.diff(hR) >= 0).all()  # nearer moves further
        assert set((hL + hR).tolist()) <= {0, -1}  # floor(s) + floor(-s)
        assert np.abs(hL).max() <= (P + 1) // 2 and np.abs(hR).max() <= (P + 1) // 2
        if P == 0:
            assert not hL.any() and not hR.any()
    hL, hR = oracle.disparity_lut(1, P, 150)
    assert hL[0] == 0 and hR[0] == 0  # linear rule: zero depth, zero shift
    assert hR[255] == P // 2


# ----------------------------------------------------------------- warp, occlusion, fill
def _read_worked():
    vals = {}
    with open(os.path.join(GOLDEN, "worked_row_w8.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, *v = line.split()
                vals[k] = v
    return vals


def test_worked_row_example(oracle):
    g = _read_worked()
    P, T = int(g["P"][0]), int(g["T"][0])
    D = np.array([[int(v) for v in g["depth"]]], np.uint8)
    letters = "abcdefgh"
    img = np.zeros((1, 8, 3), np.uint8)
    for x in range(8):
        img[0, x] = (10 * x + 1, 10 * x + 2, 10 * x + 3)
    out = oracle.from_depth(img, D, oracle.params(max_parallax=P, threshold=T),
                            want=("left", "right", "anaglyph"))
    for view in ("left", "right"):
        expect = np.array([img[0, letters.index(c)] for c in g[view]])
        assert np.array_equal(out[view][0], expect), view
    ana = np.concatenate([out["left"][..., :1], out["right"][..., 1:]], axis=-1)
    assert np.array_equal(out["anaglyph"], ana)


@pytest.mark.parametrize("rule", [0, 1])
def test_zero_parallax_gives_identical_views(oracle, rule):
    rng = np.random.default_rng(2)
    img = rng_img(rng, 23, 37)
    out = oracle.dibr(img, oracle.params(max_parallax=0, disparity_rule=rule),
                      want=("left", "right", "anaglyph"))
    assert np.array_equal(out["left"], img) and np.array_equal(out["right"], img)
    assert np.array_equal(out["anaglyph"], img)


def test_linear_rule_zero_depth_gives_identical_views(oracle):
    rng = np.random.default_rng(3)
    img = rng_img(rng, 11, 29)
    D = np.zeros((11, 29), np.uint8)
    out = oracle.from_depth(img, D, oracle.params(max_parallax=64, disparity_rule=1),
                            want=("left", "right"))
    assert np.array_equal(out["left"], img) and np.array_equal(out["right"], img)


@pytest.mark.parametrize("d", [0, 40, 150, 151, 200, 255])
@pytest.mark.parametrize("rule", [0, 1])
def test_constant_depth_is_uniform_shift(oracle, d, rule):
    rng = np.random.default_rng(4 + d)
    H, W, P = 5, 50, 24
    img = rng_img(rng, H, W)
    D = np.full((H, W), d, np.uint8)
    out = oracle.from_depth(img, D, oracle.params(max_parallax=P, disparity_rule=rule),
                            want=("left", "right"))
    hL, hR = oracle.disparity_lut(rule, P, 150)
    for view, h in (("left", int(hL[d])), ("right", int(hR[d]))):
        o = out[view]
        for t in range(W):
            s = t + h  # the source that lands on t
            if abs(h) >= W:
                s = t  # nothing lands in the row: the input pixel stays
            elif not 0 <= s < W:
                # border hole: only one side has filled targets, and the nearest one
                # shows the edge column of the source row
                s = min(max(s, 0), W - 1)
            assert np.array_equal(o[:, t], img[:, s]), (view, t)


def test_hole_runs_get_one_colour(oracle):
    rng = np.random.default_rng(5)
    for _ in range(20):
        W = 64
        D = np.repeat(rng.integers(0, 256, size=8, dtype=np.uint8), 8)[None]
        img = rng_img(rng, 1, W)
        hL, hR = oracle.disparity_lut(0, 32, 150)
        out = oracle.from_depth(img, D, oracle.params(max_parallax=32), want=("left", "right"))
        for view, h in (("left", hL), ("right", hR)):
            covered = np.zeros(W, bool)
            for x in range(W):
                t = x - int(h[D[0, x]])
                if 0 <= t < W:
                    covered[t] = True
            t = 0
            while t < W:
                if covered[t]:
                    t += 1
                    continue
                u = t
                while u < W and not covered[u]:
                    u += 1
                run = out[view][0, t:u]
                assert (run == run[0]).all()
                t = u


def test_occlusion_winner_is_extreme_source(oracle):
    # monotone tables: on every collision the left view keeps the smallest source column
    # and the right view the largest (nearer pixels are further along the shift)
    rng = np.random.default_rng(6)
    W = 40
    for _ in range(30):
        D = rng.integers(0, 256, size=(1, W), dtype=np.uint8)
        img = np.zeros((1, W, 3), np.uint8)
        img[0, :, 0] = np.arange(W)  # colour encodes the source column
        img[0, :, 1] = 7
        hL, hR = oracle.disparity_lut(0, 20, 150)
        out = oracle.from_depth(img, D, oracle.params(max_parallax=20), want=("left", "right"))
        for view, h, pick in (("left", hL, min), ("right", hR, max)):
            for t in range(W):
                srcs = [x for x in range(W) if x - int(h[D[0, x]]) == t]
                if srcs:
                    assert out[view][0, t, 0] == pick(srcs)


# ---------------------------------------------------------------------------- formatting
def test_anaglyph_and_hsbs_closed_forms(oracle):
    rng = np.random.default_rng(7)
    img = rng_img(rng, 17, 42)
    out = oracle.dibr(img, oracle.params(max_parallax=12),
                      want=("anaglyph", "left", "right", "hsbs", "depth"))
    L, R = out["left"].astype(int), out["right"].astype(int)
    assert np.array_equal(out["anaglyph"][..., 0], out["left"][..., 0])
    assert np.array_equal(out["anaglyph"][..., 1:], out["right"][..., 1:])
    sq = lambda V: (V[:, 0::2] + V[:, 1::2] + 1) // 2
    assert np.array_equal(out["hsbs"], np.concatenate([sq(L), sq(R)], axis=1).astype(np.uint8))
    Y = oracle.luma(img)
    assert np.array_equal(out["depth"], oracle.smooth_binom5(Y))


def test_rejects_odd_width_hsbs(oracle):
    img = np.zeros((2, 5, 3), np.uint8)
    with pytest.raises(ValueError):
        oracle.dibr(img, oracle.params(), want=("hsbs",))


def test_band_driver_matches_whole_image(oracle):
    rng = np.random.default_rng(8)
    img = rng_img(rng, 37, 33)
    for depth_rule in (0, 1, 2):
        p = oracle.params(max_parallax=10, depth_rule=depth_rule)
        full = oracle.dibr(img, p, want=("left", "right", "depth"))
        for y0, y1 in [(0, 1), (0, 5), (3, 9), (30, 37), (36, 37), (0, 37)]:
            part = oracle.dibr_rows(img, p, y0, y1, want=("left", "right", "depth"))
            for k in full:
                assert np.array_equal(part[k][y0:y1], full[k][y0:y1]), (depth_rule, y0, y1, k)


# ------------------------------------------------------ brute force against naive twin
def _naive_arrays(res):
    return {k: np.array(v, dtype=np.uint8) for k, v in res.items()}


@pytest.mark.parametrize("P", [0, 1, 2, 3, 4, 16])
def test_naive_twin_random_8x8(oracle, P):
    rng = np.random.default_rng(100 + P)
    for seed in range(12):
        img = rng_img(rng, 8, 8)
        for rule, rname in ((0, "paper"), (1, "linear")):
            for dr, dname in ((1, "binom5"), (0, "luma")):
                p = oracle.params(max_parallax=P, disparity_rule=rule, depth_rule=dr)
                got = oracle.dibr(img, p, want=("left", "right", "anaglyph", "hsbs", "depth"))
                ref = _naive_arrays(naive.pipeline(img.tolist(), P, 150, rname, dname))
                for k in got:
                    assert np.array_equal(got[k], ref[k]), (P, seed, rname, dname, k)


@pytest.mark.parametrize("P", [0, 1, 2, 3, 4, 16])
def test_naive_twin_gather_mode(oracle, P):
    rng = np.random.default_rng(200 + P)
    for seed in range(8):
        img = rng_img(rng, 6, 8)
        p = oracle.params(max_parallax=P, warp_mode=1)
        got = oracle.dibr(img, p, want=("left", "right", "anaglyph"))
        ref = _naive_arrays(naive.pipeline(img.tolist(), P, 150, "paper", "binom5", mode="gather"))
        for k in got:
            assert np.array_equal(got[k], ref[k]), (P, seed, k)


@pytest.mark.parametrize("P", [1, 4, 16, 64])
def test_naive_twin_every_depth_value(oracle, P):
    # one row carrying all 256 depth values in a shuffled order, several permutations
    rng = np.random.default_rng(300 + P)
    for _ in range(3):
        D = rng.permutation(256).astype(np.uint8)[None]
        img = rng_img(rng, 1, 256)
        for rule, rname in ((0, "paper"), (1, "linear")):
            for mode, mname in ((0, "forward"), (1, "gather")):
                if mode == 1 and rule == 1:
                    continue
                p = oracle.params(max_parallax=P, disparity_rule=rule, warp_mode=mode)
                got = oracle.from_depth(img, D, p, want=("left", "right"))
                ref = naive.pipeline(img.tolist(), P, 150, rname, mode=mname, D=D.tolist())
                for k in ("left", "right"):
                    assert np.array_equal(got[k], np.array(ref[k], np.uint8)), (P, rname, mname, k)


def test_gather_mode_out_of_range_falls_back_to_own_pixel(oracle):
    # Fig. 3: a sample position outside the row copies the pixel at the target itself
    img = np.arange(3 * 6, dtype=np.uint8).reshape(1, 6, 3)
    D = np.zeros((1, 6), np.uint8)  # s_L = +P/2 = +4: x + 4 is in range only for x <= 1
    out = oracle.from_depth(img, D, oracle.params(max_parallax=8, warp_mode=1), want=("left", "right"))
    assert out["left"][0].tolist() == [img[0, 4].tolist(), img[0, 5].tolist()] + img[0, 2:].tolist()
    assert out["right"][0].tolist() == img[0, :4].tolist() + [img[0, 0].tolist(), img[0, 1].tolist()]


def test_gather_mode_truncates_toward_zero(oracle):
    # s_L(151) with P = 1 is -151/510: x = 0 samples int(-0.296) = 0 (in range), where a
    # floored shift would fall off the row; Fig. 3's (int) cast truncates
    img = np.array([[[9, 9, 9], [50, 60, 70]]], np.uint8)
    D = np.array([[151, 0]], np.uint8)
    out = oracle.from_depth(img, D, oracle.params(max_parallax=1, warp_mode=1), want=("left",))
    assert out["left"][0, 0].tolist() == [9, 9, 9]


# ------------------------------------------------------------------ cross-bilateral filter
def test_xbf_constant_image_unchanged(oracle):
    img = np.full((9, 12, 3), (40, 90, 200), np.uint8)
    Y = oracle.luma(img)
    assert np.array_equal(oracle.smooth_xbf(img, Y, 2, 1.5, 16.0), Y)


@pytest.mark.parametrize("r,ss", [(1, 0.8), (2, 1.5), (3, 2.0)])
def test_xbf_large_range_sigma_is_normalised_gaussian(oracle, r, ss):
    # sigma_r -> infinity leaves the spatial Gaussian over the clipped window:
    # D = correlate(Y, G) / correlate(1, G) with zero padding outside the image
    rng = np.random.default_rng(9 + r)
    img = rng_img(rng, 14, 19)
    Y = oracle.luma(img)
    ax = np.arange(-r, r + 1)
    G = np.exp(-(ax[:, None] ** 2 + ax[None, :] ** 2) / (2 * ss * ss))
    num = ndimage.correlate(Y.astype(np.float64), G, mode="constant", cval=0.0)
    den = ndimage.correlate(np.ones_like(Y, np.float64), G, mode="constant", cval=0.0)
    v = num / den
    got = oracle.smooth_xbf(img, Y, r, ss, 1e9)
    safe = np.abs(v - np.floor(v) - 0.5) > 1e-6
    assert np.array_equal(got[safe], np.floor(v[safe] + 0.5).astype(np.uint8))
    assert safe.mean() > 0.99


def test_xbf_small_range_sigma_keeps_edges(oracle):
    # two flat regions: with a tiny range sigma the other region's weight underflows to
    # zero, so every pixel keeps its own region's luminance (the edge is not blurred)
    img = np.zeros((8, 10, 3), np.uint8)
    img[:, :5] = (200, 30, 30)
    img[:, 5:] = (20, 40, 220)
    Y = oracle.luma(img)
    assert np.array_equal(oracle.smooth_xbf(img, Y, 2, 1.5, 0.5), Y)
    # with a huge range sigma the same edge is blurred
    assert not np.array_equal(oracle.smooth_xbf(img, Y, 2, 1.5, 1e9), Y)


def test_xbf_brute_force_tiny(oracle):
    rng = np.random.default_rng(10)
    img = rng_img(rng, 5, 6)
    Y = oracle.luma(img)
    r, ss, sr = 2, 1.5, 16.0
    got = oracle.smooth_xbf(img, Y, r, ss, sr)
    for y in range(5):
        for x in range(6):
            num = den = 0.0
            for qy in range(max(0, y - r), min(5, y + r + 1)):
                for qx in range(max(0, x - r), min(6, x + r + 1)):
                    dc = img[y, x].astype(float) - img[qy, qx].astype(float)
                    w = math.exp(-((qx - x) ** 2 + (qy - y) ** 2) / (2 * ss * ss)
                                 - float(dc @ dc) / (2 * sr * sr))
                    num += w * int(Y[qy, qx])
                    den += w
            v = num / den
            if abs(v - math.floor(v) - 0.5) > 1e-9:
                assert got[y, x] == math.floor(v + 0.5), (y, x)



def test_fill_comes_from_the_farther_side_of_a_depth_edge(oracle):
    # one depth edge per row (two flat regions): every hole that has filled targets on
    # both sides shows the colour of a source from the farther (smaller depth) region --
    # the background-side reading of the fill, which the directional rule implements
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(300):
        W = int(rng.integers(8, 80))
        e = int(rng.integers(1, W))
        d1, d2 = (int(v) for v in rng.integers(0, 256, 2))
        if d1 == d2:
            continue
        D = np.array([[d1] * e + [d2] * (W - e)], np.uint8)
        img = np.zeros((1, W, 3), np.uint8)
        img[0, :, 0] = np.arange(W)  # colour encodes the source column
        P, rule = int(rng.integers(1, 96)), int(rng.integers(0, 2))
        out = oracle.from_depth(img, D, oracle.params(max_parallax=P, disparity_rule=rule), want=("left", "right"))
        hL, hR = oracle.disparity_lut(rule, P, 150)
        for view, h in (("left", hL), ("right", hR)):
            covered = np.zeros(W, bool)
            for x in range(W):
                t = x - int(h[D[0, x]])
                if 0 <= t < W:
                    covered[t] = True
            idx = np.flatnonzero(covered)
            for t in np.flatnonzero(~covered):
                if idx.size and idx[0] < t < idx[-1]:
                    src = int(out[view][0, t, 0])
                    assert D[0, src] == min(d1, d2), (view, W, e, d1, d2, P, rule, t)
                    checked += 1
    assert checked > 100
