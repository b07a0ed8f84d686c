"""Deliberately naive pure-Python restatement of the pipeline -- TEST INFRASTRUCTURE ONLY.

It shares no code with the C oracle and is written in a different formulation, so that
the two cross-check each other on tiny images:
  * rational arithmetic (``fractions.Fraction``) instead of integer tricks;
  * the depth filter as one direct 5 x 5 sum instead of two separable passes;
  * occlusion by listing every source that lands on a target and taking the best one,
    instead of a running z-buffer;
  * hole fill by listing all filled targets to each side, instead of walking;
  * the 2-D inpainting on a dictionary of the damaged pixels and a full copy of the frame
    per block, instead of a bordered block matrix.
Sections of the paper followed: Sec. 3 (six components), Sec. 4 (stage list), Fig. 3
(shift rule, threshold, out-of-range fallback, red-cyan channel map).
"""
import math
from fractions import Fraction

HALF = Fraction(1, 2)


def luma(img):
    """Depth map (Sec. 3): BT.601 luminance 0.299 R + 0.587 G + 0.114 B, rounded half up."""
    H, W = len(img), len(img[0])
    return [[math.floor(Fraction(299, 1000) * int(img[y][x][0]) + Fraction(587, 1000) * int(img[y][x][1])
                        + Fraction(114, 1000) * int(img[y][x][2]) + HALF)
             for x in range(W)] for y in range(H)]


def binom5(Y):
    """Filtered depth map, default smoothing: 2-D binomial weights b_i*b_j/256, clamped
    coordinates, rounded half up (one direct 25-tap sum)."""
    H, W = len(Y), len(Y[0])
    b = [1, 4, 6, 4, 1]
    out = []
    for y in range(H):
        row = []
        for x in range(W):
            s = Fraction(0)
            for i in range(5):
                for j in range(5):
                    yy = min(max(y + i - 2, 0), H - 1)
                    xx = min(max(x + j - 2, 0), W - 1)
                    s += Fraction(b[i] * b[j], 256) * Y[yy][xx]
            row.append(math.floor(s + HALF))
        out.append(row)
    return out


def shift_left(d, P, T, rule):
    """s_L(d) of Fig. 3 as an exact rational (rule 'paper'), or the linear alternative."""
    if rule == "paper":
        if d > T:
            return -Fraction(P, 2) * Fraction(d, 255)
        return Fraction(P, 2) * (1 - Fraction(d, 255))
    # linear: magnitude floor(P d / 510), nearer pixels move right in the left view
    return -Fraction(math.floor(Fraction(P * d, 510)))


def luts(P, T, rule):
    hL = [math.floor(shift_left(d, P, T, rule)) for d in range(256)]
    if rule == "paper":
        hR = [math.floor(-shift_left(d, P, T, rule)) for d in range(256)]
    else:
        hR = [-v for v in hL]
    return hL, hR


def forward_view(Drow, h, left):
    """Source column shown at each target of one row (forward warp, occlusion, row fill)."""
    W = len(Drow)
    winner = [None] * W
    for t in range(W):
        cands = [x for x in range(W) if x - h[Drow[x]] == t]
        if cands:
            # nearest = largest depth; equal depth: smaller x (left view), larger x (right)
            winner[t] = max(cands, key=lambda x: (Drow[x], -x if left else x))
    src = []
    for t in range(W):
        if winner[t] is not None:
            src.append(winner[t])
            continue
        lefts = [u for u in range(t) if winner[u] is not None]
        rights = [u for u in range(t + 1, W) if winner[u] is not None]
        if lefts and rights:
            l, r = lefts[-1], rights[0]
            pick = l if Drow[winner[l]] <= Drow[winner[r]] else r
            src.append(winner[pick])
        elif lefts:
            src.append(winner[lefts[-1]])
        elif rights:
            src.append(winner[rights[0]])
        else:
            src.append(t)
    return src


def gather_view(Drow, P, T, left):
    """Fig. 3 literally: sample column int(x + s) (truncation toward zero), or x itself."""
    W = len(Drow)
    src = []
    for x in range(W):
        s = shift_left(Drow[x], P, T, "paper")
        if not left:
            s = -s
        xs = int(x + s)  # int() of a Fraction truncates toward zero, like C's (int) cast
        src.append(xs if 0 <= xs < W else x)
    return src


def pipeline(img, P, T=150, rule="paper", depth="binom5", mode="forward", D=None):
    """Whole pipeline on a tiny image (list or array H x W x 3).  Returns dict of
    outputs as nested lists: depth, left, right, anaglyph, hsbs (if W even)."""
    H, W = len(img), len(img[0])
    if D is None:
        Y = luma(img)
        D = binom5(Y) if depth == "binom5" else Y
    D = [[int(v) for v in row] for row in D]
    hL, hR = luts(P, T, rule)
    left, right = [], []
    for y in range(H):
        if mode == "forward":
            sL = forward_view(D[y], hL, True)
            sR = forward_view(D[y], hR, False)
        else:
            sL = gather_view(D[y], P, T, True)
            sR = gather_view(D[y], P, T, False)
        left.append([[int(img[y][sL[t]][c]) for c in range(3)] for t in range(W)])
        right.append([[int(img[y][sR[t]][c]) for c in range(3)] for t in range(W)])
    ana = [[[left[y][t][0], right[y][t][1], right[y][t][2]] for t in range(W)] for y in range(H)]
    out = dict(depth=D, left=left, right=right, anaglyph=ana)
    if W % 2 == 0:
        half = W // 2
        hsbs = []
        for y in range(H):
            row = []
            for x in range(W):
                v, k = (left[y], x) if x < half else (right[y], x - half)
                row.append([math.floor(Fraction(v[2 * k][c] + v[2 * k + 1][c], 2) + HALF)
                            for c in range(3)])
            hsbs.append(row)
        out["hsbs"] = hsbs
    return out


def inpaint2d(view, damaged, block):
    """Fig. 3's iterative block inpainting: per block a private copy of the whole frame;
    damaged pixels listed block-column by block-column; passes over the list repair every
    damaged pixel with >= 2 undamaged 8-neighbours (mean rounded half up, visible at once
    to later pixels of the pass) until none is left or a pass repairs nothing."""
    H, W = len(view), len(view[0])
    out = [[list(map(int, view[y][x])) for x in range(W)] for y in range(H)]
    left = 0
    for by in range(0, H, block):
        for bx in range(0, W, block):
            frame = [[list(map(int, view[y][x])) for x in range(W)] for y in range(H)]
            dmg = {(x, y): bool(damaged[y][x]) for y in range(H) for x in range(W)}
            order = [(x, y) for x in range(bx, min(bx + block, W)) for y in range(by, min(by + block, H))
                     if dmg[(x, y)]]
            todo = len(order)
            while todo:
                fixed = 0
                for (x, y) in order:
                    if not dmg[(x, y)]:
                        continue
                    good = [(x + dx, y + dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                            if (dx or dy) and 0 <= x + dx < W and 0 <= y + dy < H and not dmg[(x + dx, y + dy)]]
                    if len(good) < 2:
                        continue
                    dmg[(x, y)] = False
                    todo -= 1
                    fixed += 1
                    frame[y][x] = [math.floor(Fraction(sum(frame[v][u][c] for (u, v) in good), len(good)) + HALF)
                                   for c in range(3)]
                if not fixed:
                    break
            left += todo
            for y in range(by, min(by + block, H)):
                for x in range(bx, min(bx + block, W)):
                    out[y][x] = frame[y][x]
    return out, left
