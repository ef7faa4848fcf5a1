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


def _warp_sum10(v):
    """The backward kernel's reduce-scatter of ten values over 32 lanes: four halving
    exchanges (xor 16, 8, 4, 2) each keeping one half of the values and adding the partner's
    copy of it, then a final exchange with xor 1."""
    lanes = np.arange(32)
    cur = v.copy()
    for d, keep in ((16, 5), (8, 3), (4, 2), (2, 1)):
        n = cur.shape[1]
        pad = 2 * keep - n
        if pad > 0:
            cur = np.concatenate([cur, np.zeros((32, pad))], axis=1)
        hi = (lanes & d) != 0
        lo_part, hi_part = cur[:, :keep], cur[:, keep:2 * keep]
        mine = np.where(hi[:, None], hi_part, lo_part)
        give = np.where(hi[:, None], lo_part, hi_part)          # what this lane sends
        cur = mine + give[lanes ^ d]
    y = cur[:, 0]
    return y + y[lanes ^ 1]


def test_reduce_scatter_lane_layout():
    """After the 12 shuffles, lanes 2m and 2m + 1 hold the warp sum of value j = 5 b4 + s,
    s = 3 b3 + 2 b2 + b1 (b_k the lane bits), valid when s <= 2 (b3 = 0) or s <= 4
    (b3 = 1); the kernel issues its atomic for term j from exactly those even lanes, so every
    term is added once."""
    rng = np.random.default_rng(0)
    for _ in range(50):
        v = rng.normal(size=(32, 10))
        tot = _warp_sum10(v)
        ref = v.sum(axis=0)
        seen = []
        for L in range(32):
            b4, b3, b2, b1 = (L >> 4) & 1, (L >> 3) & 1, (L >> 2) & 1, (L >> 1) & 1
            s = 3 * b3 + 2 * b2 + b1
            if (L & 1) == 0 and s <= (4 if b3 else 2):
                j = 5 * b4 + s
                assert abs(tot[L] - ref[j]) < 1e-9, (L, j)
                seen.append(j)
        assert sorted(seen) == list(range(10))


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
