"""The visiting schedule of the GPU 2-D inpainting kernel, modelled in plain Python, against
the oracle's sequential passes (Fig. 3, left column).  CPU only.

The kernel runs the figure's passes pipelined in one wavefront: pass p visits block pixel
(x, y) at step 2x + y + 4p, the visits of one step are made independently, a damaged pixel
is visited only while "dirty" (never visited, or next to a repair since its last visit),
steps without such a pixel are skipped, and the block is done when no damaged pixel is
dirty.  This model follows those rules (not the kernel's code) and must give the oracle's
result exactly: the claim that the schedule reproduces the sequential visiting order.
"""
import numpy as np
import pytest

from oracle import oracle as O


def _model_block(view, dmg, bx0, by0, bw, bh):
    H, W = dmg.shape
    flag, cell = {}, {}
    for j in range(bh + 2):
        for i in range(bw + 2):
            x, y = bx0 - 1 + i, by0 - 1 + j
            bad = not (0 <= x < W and 0 <= y < H) or dmg[y, x] != 0
            flag[i, j] = bad
            cell[i, j] = (0, 0, 0) if bad else tuple(int(c) for c in view[y, x])
    dirty = {(i, j) for i in range(1, bw + 1) for j in range(1, bh + 1) if flag[i, j]}

    def visit(i, j, new):
        nb = [(i + di, j + dj) for dj in (-1, 0, 1) for di in (-1, 0, 1) if di or dj]
        n = sum(1 for q in nb if not flag[q])
        if n < 2:
            return False
        s = [sum(cell[q][c] for q in nb) for c in range(3)]
        new[i, j] = tuple((2 * sc + n) // (2 * n) for sc in s)
        return True

    t = 0
    while True:
        # the next step at which some column has a dirty damaged pixel to visit: per column,
        # max(t, 2x + its lowest dirty row) (t when it has reached one, else that row's first
        # visit)
        nxt = None
        for x in range(bw):
            rows = [j - 1 for j in range(1, bh + 1) if flag[x + 1, j] and (x + 1, j) in dirty]
            if rows:
                n = max(t, 2 * x + min(rows))
                nxt = n if nxt is None else min(nxt, n)
        if nxt is None:
            break
        t = nxt
        # every visit of step t against the state before the step (they are independent)
        new = {}
        for x in range(bw):
            b = t - 2 * x
            for y in range(bh):
                i, j = x + 1, y + 1
                if 0 <= b - y and (b - y) % 4 == 0 and flag[i, j] and (i, j) in dirty:
                    dirty.discard((i, j))
                    visit(i, j, new)
        for (i, j), c in new.items():
            flag[i, j] = False
            cell[i, j] = c
        for (i, j) in new:
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    q = (i + di, j + dj)
                    if 1 <= q[0] <= bw and 1 <= q[1] <= bh and flag[q]:
                        dirty.add(q)
        t += 1
    return flag, cell


def _model(view, dmg, block):
    H, W = dmg.shape
    out = view.copy()
    for by0 in range(0, H, block):
        for bx0 in range(0, W, block):
            bw, bh = min(block, W - bx0), min(block, H - by0)
            flag, cell = _model_block(view, dmg, bx0, by0, bw, bh)
            for j in range(1, bh + 1):
                for i in range(1, bw + 1):
                    if dmg[by0 + j - 1, bx0 + i - 1] and not flag[i, j]:
                        out[by0 + j - 1, bx0 + i - 1] = cell[i, j]
    return out


@pytest.mark.parametrize("seed", range(12))
def test_pipelined_passes_equal_the_sequential_passes(seed):
    rng = np.random.default_rng(seed)
    W, H = int(rng.integers(1, 30)), int(rng.integers(1, 30))
    block = int(rng.choice([2, 3, 4, 8, 16, 32]))
    view = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    dmg = (rng.random((H, W)) < rng.random()).astype(np.uint8)
    out, _ = O.inpaint2d(view, dmg, block)
    assert np.array_equal(_model(view, dmg, block), out)


@pytest.mark.parametrize("side", ["left", "right"])
def test_pipelined_passes_wide_hole_repaired_one_column_per_pass(side):
    # a hole across most of the block with its only undamaged side to the right: the
    # sequential passes repair one column each, the case the pipelining exists for
    rng = np.random.default_rng(7)
    H, W = 16, 16
    view = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    dmg = np.zeros((H, W), np.uint8)
    if side == "left":
        dmg[:, :13] = 1
    else:
        dmg[:, 3:] = 1
    out, left = O.inpaint2d(view, dmg, 16)
    assert left == 0
    assert np.array_equal(_model(view, dmg, 16), out)
