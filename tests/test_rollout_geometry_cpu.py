"""Host-side check of the whole-rollout kernel's tiling assumptions for every
grid its eligibility rule admits (C = 128 and 4 heads aside): H % 8 == 0,
W % 16 == 0, W >= 32, latitude and longitude windows of at most 5, and every
8-row patch's latitude halo spanning 8 to 12 rows.

The kernel gives each CTA an 8 x 16 (latitude x longitude) query patch and
stages, per key level, a slab of the patch's halo: latitudes S0 .. S0 + SR - 1
(the union of the patch rows' clamped windows) x 20 longitudes from w0 - 2
(wrapped). Each warp takes a 4 x 4 query group and reads an 8 x 8 key
rectangle of that slab: slab rows R0 .. R0 + 7 with R0 = min(start of its
first query row's window - S0, SR - 8), slab columns 4 gc .. 4 gc + 7. The
windows are the paper's bump windows (App. A.2): start = clamp(i - k // 2,
0, n - k) in latitude, periodic and centred in longitude. This test walks
every such grid up to 96 latitudes and checks, query by query, that the
window lies inside the warp's rectangle, that the rectangle lies inside the
slab and the slab inside the grid, and that a slab never holds a longitude
twice; and that the eligibility rule admits exactly the latitude counts for
which the halo condition holds.
"""
import pytest

TH, TW, SW, SR_MAX = 8, 16, 20, 12


def clamp(v, lo, hi):
    return max(lo, min(v, hi))


def start(i, k, n):
    return clamp(i - k // 2, 0, n - k)


def halo_rows(H, kh, h0):
    S0 = start(h0, kh, H)
    return S0, start(h0 + TH - 1, kh, H) + kh - S0


def eligible(H, W, kh, kw):
    if H % 8 or W % 16 or W < 32 or kh > 5 or kw > 5 or kh > H:
        return False
    return all(8 <= halo_rows(H, kh, h0)[1] <= 12 for h0 in range(0, H, TH))


@pytest.mark.parametrize("kh", [1, 3, 5])
def test_latitude_rectangles_hold_every_window(kh):
    admitted = 0
    for H in range(8, 97, 8):
        if not eligible(H, 48, kh, 5):
            continue
        admitted += 1
        for h0 in range(0, H, TH):
            S0, SR = halo_rows(H, kh, h0)
            assert 0 <= S0 and S0 + SR <= H and 8 <= SR <= SR_MAX
            for gr in (0, 1):
                R0 = min(start(h0 + 4 * gr, kh, H) - S0, SR - 8)
                assert 0 <= R0 and R0 + 8 <= SR, (H, kh, h0, gr)
                for q in range(h0 + 4 * gr, h0 + 4 * gr + 4):
                    s = start(q, kh, H) - S0 - R0          # first rectangle row of q's window
                    assert 0 <= s and s + kh <= 8, (H, kh, h0, q)
    assert admitted >= 10   # every multiple of 8 from 8 to 96 (kh <= 5 <= H)


@pytest.mark.parametrize("kw", [1, 3, 5])
def test_longitude_rectangles_hold_every_window_without_repeats(kw):
    for W in range(32, 385, 16):
        for w0 in range(0, W, TW):
            slab = [(w0 - 2 + c) % W for c in range(SW)]
            assert len(set(slab)) == SW, (W, w0)           # no longitude twice in a slab
            for gc in range(4):
                rect = slab[4 * gc:4 * gc + 8]
                for qc in range(4):
                    q = w0 + 4 * gc + qc
                    window = {(q + d) % W for d in range(-(kw // 2), kw // 2 + 1)}
                    assert window <= set(rect), (W, w0, gc, qc)
                    # the kernel's column mask: key column j of the rectangle is
                    # in q's window iff |j - 2 - qc| <= kw // 2
                    mask = {rect[j] for j in range(8) if abs(j - 2 - qc) <= kw // 2}
                    assert mask == window, (W, w0, gc, qc)


def test_wrapping_patches_split_into_two_boxes():
    """Where the halo wraps (w0 = 0, or w0 = W - 16), the slab is two boxes:
    longitudes W-2, W-1 then 0..17, or W-18..W-1 then 0, 1; both in the grid."""
    for W in range(32, 385, 16):
        for w0 in range(0, W, TW):
            slab = [(w0 - 2 + c) % W for c in range(SW)]
            if w0 == 0:
                assert slab[:2] == [W - 2, W - 1] and slab[2:] == list(range(18))
            elif w0 + TW + 2 > W:
                assert w0 == W - 16
                assert slab[:18] == list(range(W - 18, W)) and slab[18:] == [0, 1]
            else:
                assert slab == list(range(w0 - 2, w0 + 18))
