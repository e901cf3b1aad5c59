"""Pins of the oracle's extensions: Alg. 1's ZERO-PAD search window (Alg. 1,
Sec. 3.6), the two-stage rigid search (Sec. 3.6), NMI (Sec. 2.1), SWMI (Sec. 3.3) and
label volumes.

Each pin ties the oracle to something other than itself: the unpadded direct
CMIF at the same displacement (padding with mask 0 adds no pixel pairs), the
overlap-area bound of the gamma gate for full masks, the label entropy of a
template cut out of A (MI(chi*) = H(B), Sec. 2), the strict-greater rule
of Alg. 1 across the two stages, and NMI's closed forms (2 for A = B, 1 for
independent labels).
"""
import math

import numpy as np
import pytest

import oracle

scipy_stats = pytest.importorskip("scipy.stats")


def _labels(rng, H, W, K):
    A = rng.integers(0, K, (H, W)).astype(np.int32)
    A[: H // 2, : W // 2] = 0          # some structure so that maps have a clear peak
    A[H // 2:, W // 2:] = K - 1
    return A


@pytest.mark.parametrize("shapes", [((10, 12), (10, 12)), ((13, 11), (7, 6)), ((9, 9), (9, 5))])
@pytest.mark.parametrize("gamma", [0.0, 0.3, 0.75])
def test_padded_window_equals_unpadded_cmif(shapes, gamma):
    """Inside X_S the padded pair's CMIF and N equal the unpadded pair's at the same chi."""
    rng = np.random.default_rng(5)
    (HA, WA), (HB, WB) = shapes
    A = _labels(rng, HA, WA, 3)
    B = rng.integers(0, 3, (HB, WB)).astype(np.int32)
    MB = (rng.random((HB, WB)) > 0.2).astype(np.uint8)
    r = oracle.alg1_padded(A, None, B, MB, 3, 3, gamma)
    full = oracle.cmif(A, None, B, MB, 3, 3)
    dy_lo, dy_hi, dx_lo, dx_hi = r["window"]
    for i, dy in enumerate(range(dy_lo, dy_hi + 1)):
        for j, dx in enumerate(range(dx_lo, dx_hi + 1)):
            if -(HA - 1) <= dy <= HB - 1 and -(WA - 1) <= dx <= WB - 1:
                assert r["sub_n"][i, j] == full["n"][dy + HA - 1, dx + WA - 1]
                assert abs(r["sub_mi"][i, j] - full["mi"][dy + HA - 1, dx + WA - 1]) < 1e-12
            else:
                assert r["sub_n"][i, j] == 0      # no overlap at all
    assert full["n"][r["dy"] + HA - 1, r["dx"] + WA - 1] == r["n"]


@pytest.mark.parametrize("gamma", [0.25, 0.5, 0.8])
def test_padded_equals_gated_full_map_for_full_masks(gamma):
    """Full masks, equal sizes: N(chi) = (H - |dy|)(W - |dx|) >= gamma H W forces
    |dy| <= H (1 - gamma) <= p_y, so the window excludes no shift that passes the
    gate, and max N (at chi = 0) lies inside it: both forms of Alg. 1 agree."""
    rng = np.random.default_rng(9)
    A = _labels(rng, 14, 12, 4)
    B = np.roll(A, (2, -3), axis=(0, 1))
    B[rng.random(B.shape) < 0.2] = 1
    r = oracle.alg1_padded(A, None, B, None, 4, 4, gamma)
    full = oracle.cmif(A, None, B, None, 4, 4)
    idx, mi, n = oracle.gamma_argmax(full["mi"], full["n"], gamma)
    dy, dx = divmod(idx, full["mi"].shape[1])
    assert (r["dy"], r["dx"], r["n"]) == (dy - 13, dx - 11, n)
    assert r["mi"] == mi


def test_template_cut_out_of_reference():
    """B = A[y0:y0+h, x0:x0+w]: at chi = (-y0, -x0) every B pixel meets its own
    source, the joint histogram is diagonal and MI = H(B) (the label entropy of
    B, scipy); no other shift in X_S can exceed H(B)."""
    rng = np.random.default_rng(21)
    A = rng.integers(0, 5, (24, 30)).astype(np.int32)
    y0, x0, h, w = 7, 11, 9, 10
    B = A[y0:y0 + h, x0:x0 + w].copy()
    r = oracle.alg1_padded(A, None, B, None, 5, 5, 0.9)
    hb = scipy_stats.entropy(np.bincount(B.ravel(), minlength=5), base=2)
    assert (r["dy"], r["dx"]) == (-y0, -x0)
    assert abs(r["mi"] - hb) < 1e-12 and r["n"] == h * w
    # template matching: X_S spans every placement of B inside A plus p of overhang
    dy_lo, dy_hi, dx_lo, dx_hi = r["window"]
    assert dy_lo <= -(24 - h) and dy_hi >= 0 and dx_lo <= -(30 - w) and dx_hi >= 0


def test_two_stage_rules():
    rng = np.random.default_rng(3)
    A = _labels(rng, 16, 16, 3)
    B, MB = oracle.warp_nn(A, None, math.radians(50.0))
    n_grid = 8
    # no refinement draws: stage (i) alone = Alg. 1 over the grid
    best, theta = oracle.align_two_stage(A, None, B, MB, 3, 3, n_grid, [], 0.5)
    per = []
    for t in range(n_grid):
        wB, wM = oracle.warp_nn(B, MB, 2 * math.pi * t / n_grid)
        ref = oracle.cmif(A, None, wB, wM, 3, 3)
        per.append((ref["mi"], ref["n"]))
    b1, _ = oracle.align(per, 0.5)
    assert best[0] == b1[0] and best[4] == b1[2] and theta == 2 * math.pi * b1[0] / n_grid
    # u = 1/2 re-evaluates the grid winner itself: equal I_T, strict > keeps stage (i)
    best2, theta2 = oracle.align_two_stage(A, None, B, MB, 3, 3, n_grid, [0.5], 0.5)
    assert best2 == best and theta2 == theta
    # the refinement interval reaches exactly the grid neighbours of theta*: the
    # draws u = 0 and u = 1 evaluate the grid angles next to the stage (i) choice
    seen = []

    def recording_warp(Bi, Mi, th):
        seen.append(th)
        return oracle.warp_nn(Bi, Mi, th)
    oracle.align_two_stage(A, None, B, MB, 3, 3, n_grid, [0.0, 1.0], 0.5, warp=recording_warp)
    step = 2 * math.pi / n_grid
    assert len(seen) == n_grid + 2 and np.allclose(seen[:n_grid], [step * t for t in range(n_grid)], atol=1e-12)
    assert abs(seen[n_grid] - (theta - step)) < 1e-12 and abs(seen[n_grid + 1] - (theta + step)) < 1e-12
    # refinement never lowers I, and a refined winner lies within one grid step
    u = [0.05, 0.3, 0.62, 0.9, 0.77]
    best3, theta3 = oracle.align_two_stage(A, None, B, MB, 3, 3, n_grid, u, 0.5)
    assert best3[4] >= best[4]
    if best3[0] >= n_grid:
        assert abs(theta3 - theta) <= 2 * math.pi / n_grid + 1e-12


def test_nmi_closed_forms():
    """A = B: at chi = 0 the joint histogram is diagonal, H_AB = H_A = H_B, NMI = 2.
    A(y, x) = y mod 2, B(y, x) = x mod 2 on an even grid: at chi = 0 every label
    pair has probability 1/4 (independent), H_AB = 2 = H_A + H_B, NMI = 1."""
    rng = np.random.default_rng(2)
    A = rng.integers(0, 5, (15, 13)).astype(np.int32)
    r = oracle.nmi(A, None, A, None, 5, 5)
    assert abs(r["nmi"][14, 12] - 2.0) < 1e-12
    yy, xx = np.mgrid[0:12, 0:10]
    A2 = (yy % 2).astype(np.int32)
    B2 = (xx % 2).astype(np.int32)
    r2 = oracle.nmi(A2, None, B2, None, 2, 2)
    assert abs(r2["nmi"][11, 9] - 1.0) < 1e-12
    ok = r2["h_ab"] > 0
    assert np.all(r2["nmi"][ok] >= 1.0 - 1e-12) and np.all(r2["nmi"][ok] <= 2.0 + 1e-12)
    assert np.all(r2["nmi"][~ok] == 0.0)


def test_swmi_pins():
    """SWMI (Sec. 3.3): unit weights give the binary CMIF; 0/1 weights give the
    masked CMIF; scaling a weight image leaves MI unchanged (the relative
    frequencies do not change); for A = B at chi = 0 the weighted joint
    histogram is diagonal with weights w^2, so MI = the entropy of the labels
    weighted by w^2 (scipy)."""
    rng = np.random.default_rng(8)
    A = rng.integers(0, 4, (9, 11)).astype(np.int32)
    B = rng.integers(0, 3, (7, 10)).astype(np.int32)
    ref = oracle.cmif(A, None, B, None, 4, 3)
    r = oracle.swmi(A, None, B, None, 4, 3)
    assert np.abs(r["mi"] - ref["mi"]).max() < 1e-12 and np.array_equal(r["nw"], ref["n"])
    MA = (rng.random(A.shape) > 0.3).astype(np.uint8)
    MB = (rng.random(B.shape) > 0.3).astype(np.uint8)
    refm = oracle.cmif(A, MA, B, MB, 4, 3)
    rm = oracle.swmi(A, MA.astype(float), B, MB.astype(float), 4, 3)
    assert np.abs(rm["mi"] - refm["mi"]).max() < 1e-12 and np.array_equal(rm["nw"], refm["n"])
    WA = rng.random(A.shape)
    WB = rng.random(B.shape)
    r1 = oracle.swmi(A, WA, B, WB, 4, 3)
    r2 = oracle.swmi(A, 3.7 * WA, B, WB, 4, 3)
    assert np.abs(r1["mi"] - r2["mi"]).max() < 1e-12
    assert np.allclose(r2["nw"], 3.7 * r1["nw"])
    w = rng.random(A.shape) + 0.1
    rs = oracle.swmi(A, w, A, w, 4, 4)
    hw = scipy_stats.entropy(np.bincount(A.ravel(), weights=(w * w).ravel(), minlength=4), base=2)
    assert abs(rs["mi"][8, 10] - hw) < 1e-12


def test_cmif3_pins():
    """Volumes: depth 1 reproduces the 2-D C oracle (MI, N and NMI); full masks give
    N = (D - |dz|)(H - |dy|)(W - |dx|) for equal sizes; A = B at chi = 0 gives
    MI = H(A) (scipy) and NMI = 2; labels that vary along different axes are
    independent at chi = 0 (NMI = 1, MI = 0); CMIF3(chi; A, B) = CMIF3(-chi; B, A)."""
    rng = np.random.default_rng(13)
    A2 = rng.integers(0, 3, (7, 8)).astype(np.int32)
    B2 = rng.integers(0, 3, (6, 9)).astype(np.int32)
    r3 = oracle.cmif3(A2[None], None, B2[None], None, 3, 3)
    r2 = oracle.cmif(A2, None, B2, None, 3, 3)
    assert np.abs(r3["mi"] - r2["mi"]).max() < 1e-12 and np.array_equal(r3["n"], r2["n"])
    assert np.abs(r3["nmi"] - oracle.nmi(A2, None, B2, None, 3, 3)["nmi"]).max() < 1e-12
    A = rng.integers(0, 4, (3, 5, 6)).astype(np.int32)
    r = oracle.cmif3(A, None, A, None, 4, 4)
    D, H, W = A.shape
    dz = np.arange(2 * D - 1) - (D - 1)
    dy = np.arange(2 * H - 1) - (H - 1)
    dx = np.arange(2 * W - 1) - (W - 1)
    nn = ((D - np.abs(dz))[:, None, None] * (H - np.abs(dy))[None, :, None] * (W - np.abs(dx))[None, None, :])
    assert np.array_equal(r["n"], nn.reshape((2 * D - 1) * (2 * H - 1), 2 * W - 1))
    ha = scipy_stats.entropy(np.bincount(A.ravel(), minlength=4), base=2)
    assert abs(r["mi"][(D - 1) * (2 * H - 1) + H - 1, W - 1] - ha) < 1e-12
    assert abs(r["nmi"][(D - 1) * (2 * H - 1) + H - 1, W - 1] - 2.0) < 1e-12
    zz, yy, xx = np.mgrid[0:4, 0:3, 0:6]
    Az = (zz % 2).astype(np.int32)           # varies along depth only
    Bx = (xx % 2).astype(np.int32)           # varies along width only
    ri = oracle.cmif3(Az, None, Bx, None, 2, 2)
    c0 = (4 - 1) * (2 * 3 - 1) + 3 - 1
    assert abs(ri["nmi"][c0, 6 - 1] - 1.0) < 1e-12 and abs(ri["mi"][c0, 6 - 1]) < 1e-12
    pos = ri["nmi"] > 0                      # H_AB > 0; elsewhere one label only on each side: MI = 0
    assert np.all(ri["nmi"][pos] >= 1.0 - 1e-12) and np.all(ri["nmi"] <= 2.0 + 1e-12)
    assert np.all(np.abs(ri["mi"][~pos]) < 1e-12)
    B = rng.integers(0, 4, (2, 4, 7)).astype(np.int32)
    rab = oracle.cmif3(A, None, B, None, 4, 4)["mi"].reshape(D + 2 - 1, H + 4 - 1, W + 7 - 1)
    rba = oracle.cmif3(B, None, A, None, 4, 4)["mi"].reshape(2 + D - 1, 4 + H - 1, 7 + W - 1)
    assert np.abs(rab - rba[::-1, ::-1, ::-1]).max() < 1e-12
