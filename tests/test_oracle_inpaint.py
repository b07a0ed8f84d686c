"""Pins of the 2-D block inpainting oracle (Fig. 3, left column) and of the pipeline's
2-D fill mode.  CPU only."""
import numpy as np
import pytest

from oracle import naive as N
from oracle import oracle as O

GOLDEN = __import__("pathlib").Path(__file__).parent / "golden" / "inpaint_worked_3x3.txt"


def _grey(rows):
    a = np.array(rows, np.uint8)
    return np.repeat(a[:, :, None], 3, axis=2)


def _read_golden():
    lines = [l.split() for l in GOLDEN.read_text().splitlines() if l.strip() and not l.startswith("#")]
    inp, exp = lines[:3], lines[3:]
    dmg = np.array([[1 if v == "D" else 0 for v in r] for r in inp], np.uint8)
    view = _grey([[0 if v == "D" else int(v) for v in r] for r in inp])
    return view, dmg, _grey([[int(v) for v in r] for r in exp])


def test_worked_example_column_order_gauss_seidel():
    view, dmg, exp = _read_golden()
    for block in (3, 4, 32):
        out, left = O.inpaint2d(view, dmg, block)
        assert left == 0
        assert np.array_equal(out, exp), out[:, :, 0]


def test_worked_example_ignores_the_colour_under_the_holes():
    view, dmg, exp = _read_golden()
    view = view.copy()
    view[dmg != 0] = 201
    out, _ = O.inpaint2d(view, dmg, 32)
    assert np.array_equal(out, exp)


def test_two_neighbours_suffice_and_the_mean_rounds_half_up():
    for a, b, want in ((1, 2, 2), (0, 255, 128), (10, 20, 15), (7, 7, 7), (254, 255, 255)):
        view = _grey([[a, 99, b]])
        out, left = O.inpaint2d(view, np.array([[0, 1, 0]], np.uint8), 8)
        assert left == 0 and out[0, 1, 0] == want, (a, b, out[0, 1, 0])


def test_one_undamaged_neighbour_is_not_enough():
    view = _grey([[40, 77]])
    out, left = O.inpaint2d(view, np.array([[0, 1]], np.uint8), 8)
    assert left == 1 and out[0, 1, 0] == 77  # kept as it came


def test_pixels_outside_the_block_are_seen_as_they_were():
    # row 0: 10 D | D 90 ; row 1: 20 30 | 60 80 (blocks of 2 columns)
    view = _grey([[10, 0, 0, 90], [20, 30, 60, 80]])
    dmg = np.array([[0, 1, 1, 0], [0, 0, 0, 0]], np.uint8)
    out2, left2 = O.inpaint2d(view, dmg, 2)
    # left block: 10, 20, 30, 60 (the damaged pixel of the right block does not count) -> 30
    # right block: 90, 30, 60, 80 (the left block's pixel still damaged for it) -> 65
    assert left2 == 0 and list(out2[0, :, 0]) == [10, 30, 65, 90]
    out4, left4 = O.inpaint2d(view, dmg, 4)
    # one block: (1,0) -> 30 first, then (2,0) sees it: 30 + 90 + 30 + 60 + 80 = 290 / 5 -> 58
    assert left4 == 0 and list(out4[0, :, 0]) == [10, 30, 58, 90]


def test_no_damage_is_identity_and_full_damage_makes_no_progress():
    rng = np.random.default_rng(3)
    view = rng.integers(0, 256, (9, 11, 3), dtype=np.uint8)
    out, left = O.inpaint2d(view, np.zeros((9, 11), np.uint8), 4)
    assert left == 0 and np.array_equal(out, view)
    out, left = O.inpaint2d(view, np.ones((9, 11), np.uint8), 4)
    assert left == 99 and np.array_equal(out, view)


@pytest.mark.parametrize("seed", range(6))
def test_uniform_surround_repairs_to_that_colour(seed):
    rng = np.random.default_rng(seed)
    H, W = 13, 17
    dmg = (rng.random((H, W)) < 0.35).astype(np.uint8)
    view = np.empty((H, W, 3), np.uint8)
    view[...] = (12, 200, 77)
    view[dmg != 0] = rng.integers(0, 256, (int(dmg.sum()), 3), dtype=np.uint8)
    out, left = O.inpaint2d(view, dmg, int(rng.integers(1, 9)))
    changed = np.any(out != view, axis=2)
    assert not np.any(changed & (dmg == 0))  # undamaged pixels never change
    repaired = dmg.astype(bool) & np.all(out == (12, 200, 77), axis=2)
    assert int(dmg.sum()) - int(repaired.sum()) >= left
    assert np.all(out[changed] == (12, 200, 77))


@pytest.mark.parametrize("seed", range(8))
def test_matches_the_naive_statement(seed):
    rng = np.random.default_rng(100 + seed)
    H, W = int(rng.integers(1, 12)), int(rng.integers(1, 12))
    view = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    dmg = (rng.random((H, W)) < rng.choice([0.1, 0.4, 0.8])).astype(np.uint8)
    block = int(rng.integers(1, 7))
    out, left = O.inpaint2d(view, dmg, block)
    nout, nleft = N.inpaint2d(view.tolist(), dmg.tolist(), block)
    assert left == nleft
    assert np.array_equal(out, np.array(nout, np.uint8))


def test_repaired_colours_stay_within_the_undamaged_range():
    rng = np.random.default_rng(9)
    view = rng.integers(40, 90, (20, 24, 3), dtype=np.uint8)
    dmg = (rng.random((20, 24)) < 0.5).astype(np.uint8)
    view[dmg != 0] = 255
    out, _ = O.inpaint2d(view, dmg, 8)
    fixed = (dmg != 0) & np.any(out != 255, axis=2)
    assert np.all((out[fixed] >= 40) & (out[fixed] < 90))


# ---- the pipeline with the 2-D fill mode

def _scene(seed, H=24, W=40):
    rng = np.random.default_rng(seed)
    img = np.zeros((H, W, 3), np.uint8)
    img[...] = rng.integers(0, 256, 3, dtype=np.uint8)
    for _ in range(4):
        y0, x0 = rng.integers(0, H - 4), rng.integers(0, W - 6)
        img[y0:y0 + rng.integers(3, 10), x0:x0 + rng.integers(4, 14)] = rng.integers(0, 256, 3, dtype=np.uint8)
    return img


@pytest.mark.parametrize("seed", range(4))
def test_holes_output_marks_the_targets_no_source_reached(seed):
    img = _scene(seed)
    p = O.params(max_parallax=12)
    out = O.dibr(img, p, want=("holes", "depth"))
    D = out["depth"]
    hL, hR = N.luts(12, 150, "paper")
    for y in range(img.shape[0]):
        for bit, h in ((1, hL), (2, hR)):
            reached = {x - h[D[y][x]] for x in range(img.shape[1])}
            holes = [t for t in range(img.shape[1]) if t not in reached]
            got = [t for t in range(img.shape[1]) if out["holes"][y, t] & bit]
            assert got == holes, (y, bit)


@pytest.mark.parametrize("seed", range(4))
def test_2d_fill_changes_only_holes_and_equals_inpainting_of_the_row_filled_views(seed):
    img = _scene(seed)
    want = ("left", "right", "anaglyph", "hsbs", "holes")
    row = O.dibr(img, O.params(max_parallax=16), want=want)
    two = O.dibr(img, O.params(max_parallax=16, fill_mode=O.FILL_INPAINT2D, inpaint_block=8), want=want)
    assert np.array_equal(row["holes"], two["holes"])
    for name, bit in (("left", 1), ("right", 2)):
        exp, _ = O.inpaint2d(row[name], row["holes"] & bit, 8)
        assert np.array_equal(two[name], exp)
        assert not np.any(np.any(two[name] != row[name], axis=2) & ((row["holes"] & bit) == 0))
    # formatting follows the inpainted views
    assert np.array_equal(two["anaglyph"][:, :, 0], two["left"][:, :, 0])
    assert np.array_equal(two["anaglyph"][:, :, 1:], two["right"][:, :, 1:])


def test_row_bands_reject_the_2d_fill():
    img = _scene(1)
    with pytest.raises(ValueError):
        O.dibr_rows(img, O.params(fill_mode=O.FILL_INPAINT2D), 0, 8)
