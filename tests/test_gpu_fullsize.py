"""Parity at the stated sizes of the rotation search and of the uneven batch.

Rotation search: 512 x 512, K = 16, 64 angles over 360 degrees, B = A rotated
by 37.5 degrees and shifted by (-23, 61) (Alg. 1 over a rotation grid,
Sec. 3.6).  For every angle the device's MI and N maps (A's transforms computed
once and reused, the Tensor-Memory row kernel at transform width 1024) are
compared with the oracle's direct method on the device-warped B at sampled
shifts (random ones, the planted shift, the map's corners and centre): N
bit-exact, MI within MI_TOL.  The device top-5 must equal Alg. 1 run on the
host over the downloaded maps, and each of the five records must agree with
the oracle at its (angle, shift).  For a few angles the joint counts of the
debug path are compared at sampled shifts as well.

Uneven batch: the 128 pairs (sides 96 .. 1536, K in {8, 16, 24}, 4 angles
each, hole masks) at their stated sizes.  The batch's per-pair choice must
equal the single-pair plan's, the plan's device top-4 must equal Alg. 1 on the
host over its maps, and the maps must match the oracle on the device-warped B:
in full for the smallest pairs (within a budget of pixel visits) and at
sampled shifts for every other pair, all 4 angles.
"""
import numpy as np
import pytest

import oracle
import synth
from tolerances import MI_TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_14699_gb300 as cm
    from paper_2106_14699_gb300 import build
    build.build()
    cm.lib()
    return cm


def _dev(x):
    return None if x is None else torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _warp(cm, dB, dM, theta, shape):
    oB = torch.empty(shape, dtype=torch.int32, device="cuda:0")
    oM = torch.empty(shape, dtype=torch.uint8, device="cuda:0")
    cm.rotate_nn(dB, dM, theta, oB, oM)
    torch.cuda.synchronize()
    return oB.cpu().numpy(), oM.cpu().numpy()


def _sample_shifts(rng, HA, WA, HB, WB, n_random, extra=()):
    """Random displacements of the full range, plus the corners, the centre and extra ones."""
    dys = list(rng.integers(-(HA - 1), HB, n_random))
    dxs = list(rng.integers(-(WA - 1), WB, n_random))
    pts = [(-(HA - 1), -(WA - 1)), (-(HA - 1), WB - 1), (HB - 1, -(WA - 1)), (HB - 1, WB - 1), (0, 0)]
    pts += [(dy, dx) for dy, dx in extra if -(HA - 1) <= dy <= HB - 1 and -(WA - 1) <= dx <= WB - 1]
    for dy, dx in pts:
        dys.append(dy)
        dxs.append(dx)
    return np.array(dys, np.int32), np.array(dxs, np.int32)


def test_rotation512_all_64_angles_vs_oracle(cm):
    cfg = synth.make_workload("rotation-512x512-K16-64angles")
    A, B = cfg["A"], cfg["B"]
    H, W = A.shape
    K = 16
    angles = cfg["angles"]
    n_ang = len(angles)
    assert n_ang == 64 and (H, W) == (512, 512)
    R, C = 2 * H - 1, 2 * W - 1
    dA, dB = _dev(A), _dev(B)
    plan = cm.Plan(H, W, H, W, K, K, cm.FP32)
    maps = torch.empty((n_ang, R, C), dtype=torch.float64, device="cuda:0")
    nmaps = torch.empty((n_ang, R, C), dtype=torch.int32, device="cuda:0")
    topk = torch.empty(24 * 5, dtype=torch.uint8, device="cuda:0")
    plan.align_rotations(dA, None, dB, None, angles, 0.5, 5, topk, maps, n_maps=nmaps)
    st = plan.status()
    assert st[0] == "OK" and st[1] < 0.25, st
    gm, gn = maps.cpu().numpy(), nmaps.cpu().numpy()
    del maps, nmaps
    rng = np.random.default_rng(4064)
    warped = []
    worst = 0.0
    for i, th in enumerate(angles):
        wB, wM = _warp(cm, dB, None, th, B.shape)
        warped.append((wB, wM))
        dys, dxs = _sample_shifts(rng, H, W, H, W, 100, extra=[cfg["shift"]])
        ref = oracle.cmif_at(A, None, wB, wM, K, K, dys, dxs)
        r, c = dys + H - 1, dxs + W - 1
        np.testing.assert_array_equal(gn[i][r, c], ref["n"], err_msg=f"angle {i}")
        err = float(np.abs(gm[i][r, c] - ref["mi"]).max())
        worst = max(worst, err)
        assert err <= MI_TOL, (i, err)
    print(f"[rotation512] 64 angles x 106 shifts: N exact, max|dMI| = {worst:.3e}")
    # the device top-5 = Alg. 1 on the host over the device maps
    best, top = oracle.align([(gm[i], gn[i]) for i in range(n_ang)], 0.5, top_k=5)
    got = cm.peaks_from_bytes(topk, 5)
    for (ga, gdy, gdx, gnn, gmi), (ra, ridx, rmi, rn) in zip(got, top):
        rdy, rdx = divmod(ridx, C)
        assert (ga, gdy, gdx, gnn) == (ra, rdy - (H - 1), rdx - (W - 1), rn)
        assert gmi == rmi
        # and the oracle agrees at each record's (angle, shift)
        wB, wM = warped[ga]
        ref = oracle.cmif_at(A, None, wB, wM, K, K, np.array([gdy], np.int32), np.array([gdx], np.int32))
        assert int(ref["n"][0]) == gnn and abs(float(ref["mi"][0]) - gmi) <= MI_TOL
    assert got[0][0] == best[0]
    # the planted truth: a grid neighbour of 37.5 degrees, shift within 3 px
    ang_deg = np.degrees(angles[got[0][0]])
    assert min(abs(ang_deg - 33.75), abs(ang_deg - 39.375)) < 1e-9
    assert abs(got[0][1] - cfg["shift"][0]) <= 3 and abs(got[0][2] - cfg["shift"][1]) <= 3
    plan.close()
    # joint counts of the debug path at sampled shifts, for a few of the angles
    dplan = cm.Plan(H, W, H, W, K, K, cm.FP32, debug_counts=True)
    counts = torch.empty((K * K + 2 * K, R, C), dtype=torch.int32, device="cuda:0")
    mi1 = torch.empty((R, C), dtype=torch.float64, device="cuda:0")
    n1 = torch.empty((R, C), dtype=torch.int32, device="cuda:0")
    for i in (0, 6, 7, 40):
        wB, wM = warped[i]
        dplan.compute(dA, None, _dev(wB), _dev(wM), mi1, n1, counts, 0.5)
        assert dplan.status()[0] == "OK"
        dys, dxs = _sample_shifts(rng, H, W, H, W, 24, extra=[cfg["shift"]])
        ref = oracle.cmif_at(A, None, wB, wM, K, K, dys, dxs, counts=True)
        r, c = dys + H - 1, dxs + W - 1
        got_joint = counts[:K * K, r, c].cpu().numpy().T          # (shifts, K*K), a-major pairs
        np.testing.assert_array_equal(got_joint, ref["joint"], err_msg=f"angle {i}")
        np.testing.assert_array_equal(n1.cpu().numpy()[r, c], gn[i][r, c])
    dplan.close()


def test_uneven_batch_full_size_vs_oracle(cm):
    cfg = synth.make_workload("uneven-batch-128pairs")
    pairs = cfg["pairs"]
    assert len(pairs) == 128
    dev_pairs = [dict(A=_dev(p["A"]), M_A=_dev(p["M_A"]), B=_dev(p["B"]), M_B=_dev(p["M_B"]), K_A=p["K_A"],
                      K_B=p["K_B"], angles=p["angles"], gamma=0.5) for p in pairs]
    batch = cm.Batch(dev_pairs, cm.FP32, graph=False)
    res = torch.empty(24 * len(pairs), dtype=torch.uint8, device="cuda:0")
    stat = torch.full((len(pairs),), -1, dtype=torch.int32, device="cuda:0")
    batch.run(res, stat)
    torch.cuda.synchronize()
    assert batch.status()[0] == "OK"
    assert stat.cpu().tolist() == [0] * len(pairs)
    got = cm.peaks_from_bytes(res, len(pairs))
    batch.close()
    # full oracle maps for the cheapest pairs, within a budget of pixel visits
    cost = [p["A"].size * p["B"].size * len(p["angles"]) for p in pairs]
    full, spent = set(), 0
    for i in sorted(range(len(pairs)), key=lambda k: cost[k]):
        if spent + cost[i] > 4e10:
            break
        full.add(i)
        spent += cost[i]
    rng = np.random.default_rng(5128)
    worst, n_full, n_sampled = 0.0, 0, 0
    for i, (p, dp) in enumerate(zip(pairs, dev_pairs)):
        HA, WA = p["A"].shape
        HB, WB = p["B"].shape
        KA, KB = p["K_A"], p["K_B"]
        R, C = HA + HB - 1, WA + WB - 1
        na = len(p["angles"])
        plan = cm.Plan(HA, WA, HB, WB, KA, KB, cm.FP32)
        maps = torch.empty((na, R, C), dtype=torch.float64, device="cuda:0")
        nmaps = torch.empty((na, R, C), dtype=torch.int32, device="cuda:0")
        top = torch.empty(24 * na, dtype=torch.uint8, device="cuda:0")
        plan.align_rotations(dp["A"], dp["M_A"], dp["B"], dp["M_B"], p["angles"], 0.5, na, top, maps, n_maps=nmaps)
        st = plan.status()
        assert st[0] == "OK" and st[1] < 0.25, (i, st)
        gm, gn = maps.cpu().numpy(), nmaps.cpu().numpy()
        del maps, nmaps
        dtop = cm.peaks_from_bytes(top, na)
        assert got[i] == dtop[0], (i, got[i], dtop[0])
        best, htop = oracle.align([(gm[a], gn[a]) for a in range(na)], 0.5, top_k=na)
        for (ga, gdy, gdx, gnn, gmi), (ra, ridx, rmi, rn) in zip(dtop, htop):
            rdy, rdx = divmod(ridx, C)
            assert (ga, gdy, gdx, gnn, gmi) == (ra, rdy - (HA - 1), rdx - (WA - 1), rn, rmi), i
        for a, th in enumerate(p["angles"]):
            wB, wM = _warp(cm, dp["B"], dp["M_B"], th, (HB, WB))
            if i in full:
                ref = oracle.cmif(p["A"], p["M_A"], wB, wM, KA, KB)
                np.testing.assert_array_equal(gn[a], ref["n"], err_msg=f"pair {i} angle {a}")
                err = float(np.abs(gm[a] - ref["mi"]).max())
                n_full += 1
            else:
                dys, dxs = _sample_shifts(rng, HA, WA, HB, WB, 48, extra=[p["shift"]])
                ref = oracle.cmif_at(p["A"], p["M_A"], wB, wM, KA, KB, dys, dxs)
                r, c = dys + HA - 1, dxs + WA - 1
                np.testing.assert_array_equal(gn[a][r, c], ref["n"], err_msg=f"pair {i} angle {a}")
                err = float(np.abs(gm[a][r, c] - ref["mi"]).max())
                n_sampled += 1
            worst = max(worst, err)
            assert err <= MI_TOL, (i, a, err)
        plan.close()
    print(f"[uneven-batch] 128 pairs: {n_full} full maps, {n_sampled} sampled maps, N exact, "
          f"max|dMI| = {worst:.3e}")
