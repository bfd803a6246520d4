"""Host-side checks of two numerical choices of the FP32 back-projection gather
(`k_bp_spline`), restated here in numpy FP32 arithmetic (no GPU, no oracle):

* the piece lookup: per view, 128 equal cells of the fractional detector position f,
  each holding the piece at the cell's left end, and E = the largest number of kinks
  strictly inside one cell.  With E <= 1 the piece of f is lut[cell] plus one compare
  with the next kink; that must be the piece a search over the sorted kinks finds, in the
  same FP32 comparisons, for every f in [0, 1] (f may round up to 1.0);
* the detector coordinate: each lane forms its first pixel's coordinate from the exact
  FP32 split of the view's steps (hi parts short enough that pixel index x hi part is
  exact), and its offsets 4 i c, 8 k s are split the same way into integer and fraction,
  so slot + f stays within a few 1e-7 bins of the FP64 coordinate (Sec. 5: the kernel
  weights are smooth in f, so this error stays far below the 1e-5 parity gate).
"""
import math

import numpy as np

f32 = np.float32
NL = 128


def _lookup(sig32):
    """Cells [c, c + 1) / NL: piece at the left end, kinks strictly inside (FP32)."""
    lut = np.zeros(NL, dtype=np.int64)
    E = 0
    for c in range(NL):
        x0 = f32(c) * f32(1.0 / NL)
        x1 = f32(c + 1) * f32(1.0 / NL)
        sr = sig32[1:16]
        lut[c] = int(np.sum(sr <= x0))
        E = max(E, int(np.sum((x0 < sr) & (sr < x1))))
    return lut, E


def _search(sig32, f, Q):
    q = 0
    for step in (8, 4, 2, 1):
        if sig32[q + step] <= f:
            q += step
    return min(q, Q - 1)


def test_piece_lookup_equals_the_search():
    rng = np.random.default_rng(11)
    n_views = n_lut = 0
    for trial in range(1200):
        Q = int(rng.integers(1, 12))
        if trial % 4 == 0:
            kinks = np.sort(rng.uniform(0.0, 1.0, Q - 1))
        elif trial % 4 == 1:  # kinks on cell edges, half of them with a second kink in that cell
            cells = np.sort(rng.choice(np.arange(1, NL), size=(Q - 1 + 1) // 2, replace=False))
            second = cells[rng.uniform(size=cells.size) < 0.5] / NL + 0.25 / NL
            kinks = np.sort(np.concatenate([cells / NL, second]))[: Q - 1]
            Q = kinks.size + 1
        else:  # clustered kinks, as near the diagonal and the axes
            kinks = np.sort((rng.uniform() + rng.normal(0.0, 0.01, Q - 1)) % 1.0)
        sig32 = np.full(16, 2.0, dtype=f32)
        sig32[: Q + 1] = np.concatenate([[0.0], kinks, [1.0]]).astype(f32)
        lut, E = _lookup(sig32)
        n_views += 1
        if E > 1:
            continue  # the kernel runs the search for this view
        n_lut += 1
        fs = np.concatenate([rng.uniform(0.0, 1.0, 300).astype(f32), sig32[: Q + 1],
                             np.nextafter(sig32[: Q + 1], f32(0.0)), [f32(1.0)]])
        for f in fs[(fs >= 0) & (fs <= 1)]:
            cell = min(int(f32(f) * f32(NL)), NL - 1)
            q = lut[cell]
            q += 1 if sig32[q + 1] <= f else 0
            assert min(q, Q - 1) == _search(sig32, f, Q)
    assert n_lut > n_views // 2


def _split(v, nb):
    m, e = math.frexp(v)
    hi = math.ldexp(math.trunc(math.ldexp(m, 24 - nb)), e - (24 - nb))
    return hi, v - hi


def _max_coordinate_error(N, na, M, lam=1.0, tiles=3, seed=0):
    rng = np.random.default_rng(seed)
    nb = 1
    while (1 << nb) < (N + 63) // 64 * 64:
        nb += 1
    T = (N + 63) // 64
    worst = 0.0
    x0 = -0.5 * (N - 1)
    for a in range(0, na, max(1, na // 120)):
        th = math.pi * a / na
        c, s = math.cos(th) / lam, math.sin(th) / lam
        pz = (x0 * c + x0 * s) + 0.5 * (M - 1)
        nz = math.floor(pz)
        t5, t6 = f32(nz), f32(pz - nz)
        chi, clo = _split(c, nb)
        shi, slo = _split(s, nb)
        t7, t8, t9, t10 = f32(chi), f32(clo), f32(shi), f32(slo)
        for _ in range(tiles):
            TX0, TY0 = 64 * int(rng.integers(0, T)), 64 * int(rng.integers(0, T))
            w = np.arange(8)[:, None]
            lane = np.arange(32)[None, :]
            Xb = TX0 + 16 * (w & 3) + (lane & 3)
            Yb = TY0 + 32 * (w >> 2) + (lane >> 2)
            X, Y = Xb.astype(f32), Yb.astype(f32)
            a1, a2 = X * t7, Y * t9
            n1, n2 = np.floor(a1), np.floor(a2)
            fr = (t6 + (a1 - n1)) + ((a2 - n2) + (Y * t10 + X * t8))
            n3 = np.floor(fr)
            mb = int(t5) + n1.astype(np.int64) + n2.astype(np.int64) + n3.astype(np.int64)
            fb = (fr - n3).astype(f32)
            for k in range(4):
                hy = f32(8 * k) * t9
                fy = np.floor(hy)
                gy = f32((hy - fy) + f32(8 * k) * t10)
                for i in range(4):
                    hx = f32(4 * i) * t7
                    fx = np.floor(hx)
                    gx = f32(fb + f32((hx - fx) + f32(4 * i) * t8))
                    pl = f32(gx + gy)
                    fl = np.floor(pl)
                    f = f32(pl - fl)
                    slot = mb + int(fx) + int(fy) + fl.astype(np.int64)
                    exact = (x0 + Xb + 4 * i) * c + (x0 + Yb + 8 * k) * s + 0.5 * (M - 1)
                    worst = max(worst, float(np.abs(slot + f.astype(np.float64) - exact).max()))
    return worst


def test_fp32_detector_coordinate_error():
    for N, na, M in ((2048, 1800, 2900), (512, 720, 726), (130, 24, 200)):
        assert _max_coordinate_error(N, na, M) < 5e-7, N
