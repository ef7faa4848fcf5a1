"""Arithmetic facts the CUDA kernels rely on, checked on the CPU: exhaustively where the
domain is small, by dense sampling where it is continuous.  Each is a claim made in a
kernel's comments that the GPU parity tests would only catch indirectly."""
import numpy as np
import pytest


def test_multiply_high_division_is_exact_for_the_placement_window():
    """Pair placement divides a pair's index j within its rectangle's window part by the
    rectangle width w with umulhi(j, ceil(2^32 / w)), magic = floor((2^32 - 1) / w) + 1 for
    w > 1 (w = 1 is taken as j itself).  Window cells: j < 512; widths: w <= 256."""
    j = np.arange(512, dtype=np.uint64)
    for w in range(2, 257):
        magic = np.uint64(0xFFFFFFFF // w + 1)
        q = (j * magic) >> np.uint64(32)
        np.testing.assert_array_equal(q, j // np.uint64(w), err_msg="w = %d" % w)
        r = j - q * np.uint64(w)
        assert (r < w).all()


RED_BATCH, RED_TERMS, RED_PITCH = 3, 10, 36   # the backward kernel's shared-memory reduction


def test_backward_row_reduction_layout():
    """The backward kernel stores lane l's value of term j of batched entry e at
    row (10 e + j), column l, rows RED_PITCH floats apart; lane r then sums row r with eight
    16-byte loads and adds it to slot j' = j (j < 7) or j + 1 of the record's three
    gradient float4s.  Every (entry, term) is summed over all 32 lanes exactly once, the rows
    fit one pass of the warp, the slots skip the two padding floats (7 and 11), every row
    starts 16-byte aligned, and the eight 16-byte reads of each quarter-warp fall on
    different bank groups."""
    rng = np.random.default_rng(0)
    v = rng.normal(size=(RED_BATCH, RED_TERMS, 32))           # [entry][term][lane]
    red = np.zeros(RED_BATCH * RED_TERMS * RED_PITCH)
    for e in range(RED_BATCH):
        for jt in range(RED_TERMS):
            for lane in range(32):
                red[(e * RED_TERMS + jt) * RED_PITCH + lane] = v[e, jt, lane]
    rows = RED_BATCH * RED_TERMS
    assert rows <= 32
    slots = np.zeros((RED_BATCH, 12))
    for r in range(rows):                                     # lane r sums row r
        row = red[r * RED_PITCH: r * RED_PITCH + 32].reshape(8, 4).sum(axis=0)
        e, jt = divmod(r, RED_TERMS)
        slots[e, jt if jt < 7 else jt + 1] += row.sum()
    ref = v.sum(axis=2)
    np.testing.assert_allclose(slots[:, [0, 1, 2, 3, 4, 5, 6, 8, 9, 10]], ref, atol=1e-12)
    assert (slots[:, [7, 11]] == 0).all()
    assert (RED_PITCH * 4) % 16 == 0
    for k in range(8):                                        # 16-byte read k of every lane
        for q in range(4):                                    # quarter-warps
            groups = {((r * RED_PITCH + 4 * k) % 32) // 4 for r in range(8 * q, 8 * q + 8)}
            assert len(groups) == 8


def _conics(rng, n):
    """Positive-definite 2D conics [[a, b], [b, c]] over a wide range of shapes and scales."""
    s = np.exp(rng.uniform(np.log(0.3), np.log(80.0), size=(n, 2)))
    th = rng.uniform(0, np.pi, size=n)
    c, s_ = np.cos(th), np.sin(th)
    inv = 1.0 / s ** 2
    a = c * c * inv[:, 0] + s_ * s_ * inv[:, 1]
    b = c * s_ * (inv[:, 0] - inv[:, 1])
    cc = s_ * s_ * inv[:, 0] + c * c * inv[:, 1]
    return a, b, cc


def test_box_bound_of_the_quadratic_form():
    """max over |ex| <= hx, |ey| <= hy of a ex^2 + 2 b ex ey + c ey^2 is a hx^2 + 2|b| hx hy +
    c hy^2 (a convex function peaks at a corner), the radius of the block used by the cull."""
    rng = np.random.default_rng(1)
    a, b, c = _conics(rng, 2000)
    hx, hy = 3.5, 1.5                              # pixel-centre half-extents of an 8x4 block
    ex, ey = np.meshgrid(np.linspace(-hx, hx, 29), np.linspace(-hy, hy, 13), indexing="ij")
    ex, ey = ex.ravel(), ey.ravel()
    q = a[:, None] * ex ** 2 + 2 * b[:, None] * ex * ey + c[:, None] * ey ** 2
    r2 = a * hx * hx + 2 * np.abs(b) * hx * hy + c * hy * hy
    assert (q.max(axis=1) <= r2 * (1 + 1e-12)).all()
    np.testing.assert_allclose(q.max(axis=1), r2, rtol=1e-12)


def test_block_cull_never_drops_a_contributing_entry():
    """The warp-level cull keeps an entry when sqrt(q(centre - mu)) <= sqrt(Q) + sqrt(r2)
    (Q = 2 ln(o / alpha_min)).  By the triangle inequality of the norm sqrt(q), an entry it
    drops has q(p - mu) > Q, i.e. alpha < alpha_min, at every pixel centre of the block."""
    rng = np.random.default_rng(2)
    n = 20000
    a, b, c = _conics(rng, n)
    o = rng.uniform(1 / 255, 0.99, size=n)
    alpha_min = 1 / 255
    bx0, by0 = 0.5, 0.5                            # pixel centres 0.5 .. 7.5 and 0.5 .. 3.5
    hx, hy = 3.5, 1.5
    cx, cy = bx0 + hx, by0 + hy
    mu = np.stack([cx + rng.normal(0, 30, n), cy + rng.normal(0, 30, n)], 1)
    dx, dy = cx - mu[:, 0], cy - mu[:, 1]
    q_c = a * dx * dx + 2 * b * dx * dy + c * dy * dy
    Q = 2 * (np.log(o) - np.log(alpha_min))
    r2 = a * hx * hx + 2 * np.abs(b) * hx * hy + c * hy * hy
    keep = np.sqrt(q_c) <= np.sqrt(Q) + np.sqrt(r2)
    px, py = np.meshgrid(np.arange(8) + 0.5, np.arange(4) + 0.5, indexing="ij")
    px, py = px.ravel(), py.ravel()
    ddx = px[None, :] - mu[:, :1]
    ddy = py[None, :] - mu[:, 1:]
    q = a[:, None] * ddx ** 2 + 2 * b[:, None] * ddx * ddy + c[:, None] * ddy ** 2
    reaches = (o[:, None] * np.exp(-0.5 * q) >= alpha_min).any(axis=1)
    assert not (reaches & ~keep).any()
    assert reaches.sum() > 100 and (~keep).sum() > 1000      # both cases exercised


def test_information_gain_exponent_in_lane_offsets():
    """The compositing kernels stage an entry as C0 = k.x ex^2 + k.y ex ey + k.z ey^2 +
    log2 o, Cu = -(2 k.x ex + k.y ey), Cv = -(k.y ex + 2 k.z ey), with (ex, ey) the mean
    relative to the 8x4 block's centre; at lane offset (u, v) = (l mod 8 - 3.5, l div 8 - 1.5)
    the exponent C0 + Cu u + Cv v + k.x u^2 + k.y u v + k.z v^2 equals the quadratic form
    k.x dx^2 + k.y dx dy + k.z dy^2 + log2 o at (dx, dy) = mean - pixel centre."""
    rng = np.random.default_rng(3)
    a, b, c = _conics(rng, 500)
    log2e = 1.4426950408889634
    kx, ky, kz = -0.5 * log2e * a, -log2e * b, -0.5 * log2e * c
    lo = np.log2(rng.uniform(0.01, 1.0, 500))
    bx0, by0 = rng.uniform(0, 300, 500), rng.uniform(0, 200, 500)     # centre of the first pixel
    mx, my = bx0 + rng.uniform(-20, 27, 500), by0 + rng.uniform(-20, 23, 500)
    ccx, ccy = bx0 + 3.5, by0 + 1.5
    ex, ey = mx - ccx, my - ccy
    c0 = kx * ex * ex + ky * ex * ey + kz * ey * ey + lo
    cu, cv = -(2 * kx * ex + ky * ey), -(ky * ex + 2 * kz * ey)
    for lane in range(32):
        u, v = (lane & 7) - 3.5, (lane >> 3) - 1.5
        pw = c0 + cu * u + cv * v + kx * u * u + ky * u * v + kz * v * v
        dx, dy = mx - (bx0 + (lane & 7)), my - (by0 + (lane >> 3))
        ref = kx * dx * dx + ky * dx * dy + kz * dy * dy + lo
        np.testing.assert_allclose(pw, ref, rtol=1e-9, atol=1e-9)


def test_live_pixel_box_of_a_lane_mask():
    """The information-gain kernel bounds the block's live pixels (lane l at column l mod 8,
    row l div 8) by OR-ing the mask's four bytes for the columns and testing each byte for the
    rows; first and last set bits give the box, which holds every live pixel and is the
    smallest such box."""
    rng = np.random.default_rng(4)
    masks = list(rng.integers(1, 1 << 32, 3000, dtype=np.uint64)) + [1 << k for k in range(32)]
    for m in masks:
        m = int(m)
        cols = (m | (m >> 8) | (m >> 16) | (m >> 24)) & 0xFF
        rows = sum(1 << r for r in range(4) if (m >> (8 * r)) & 0xFF)
        x0, x1 = (cols & -cols).bit_length() - 1, cols.bit_length() - 1
        y0, y1 = (rows & -rows).bit_length() - 1, rows.bit_length() - 1
        live = [(l & 7, l >> 3) for l in range(32) if (m >> l) & 1]
        assert x0 == min(p[0] for p in live) and x1 == max(p[0] for p in live)
        assert y0 == min(p[1] for p in live) and y1 == max(p[1] for p in live)


def _order_bucket(n):
    """The binning's item-order bucket of a list of n pairs (0: the longest lists)."""
    key = 0
    if n:
        lg = n.bit_length() - 1
        two = (n >> (lg - 2)) & 3 if lg >= 2 else (n << (2 - lg)) & 3
        key = min(4 * lg + two, 63)
    return 63 - key


def test_item_order_buckets_follow_list_length():
    """Buckets never put a longer list after a shorter one, split every doubling of the
    length in four (so lists in one bucket differ by less than 25% below 2^16), and the
    lengths from 2^16 on share bucket 0."""
    b = np.array([_order_bucket(n) for n in range(1 << 17)])
    assert (np.diff(b) <= 0).all()
    assert b[0] == b[1] == 63 and b[-1] == 0 and b[1 << 16] == 0
    for lg in range(2, 16):
        assert len(set(b[1 << lg: 1 << (lg + 1)])) == 4
