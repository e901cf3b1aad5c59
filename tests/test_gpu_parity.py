"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Counts (joint C_AB^{a,b}, marginals C_A^a, C_B^b and N) must be bit-exact;
MI must be within MI_TOL of the oracle's FP64 value (tests/tolerances.py: the
epilogue sums c log2 c exactly in fixed point, each term from a log2 whose
error over every possible count is bounded by an exhaustive test); the
rounding residual of every count must stay under the 0.25 guard.
"""
import math

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


def _to(x):
    return None if x is None else torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def run_gpu(cm, A, MA, B, MB, KA, KB, prec, counts=True, gamma=0.0):
    out = cm.cmif(_to(A), _to(MA), _to(B), _to(MB), KA, KB, precision=prec, gamma=gamma, with_counts=counts)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}


def check_exact(cm, A, MA, B, MB, KA, KB, prec, gamma=0.0):
    g = run_gpu(cm, A, MA, B, MB, KA, KB, prec, counts=True, gamma=gamma)
    ref = oracle.cmif(A, MA, B, MB, KA, KB, counts=True, marginals=True)
    assert g["status"][0] == "OK", g["status"]
    assert g["status"][1] < 0.25
    np.testing.assert_array_equal(g["n"], ref["n"])
    kk = KA * KB
    np.testing.assert_array_equal(g["counts"][:kk], ref["joint"])
    np.testing.assert_array_equal(g["counts"][kk:kk + KA], ref["marg_a"])
    np.testing.assert_array_equal(g["counts"][kk + KA:], ref["marg_b"])
    err = float(np.abs(g["mi"] - ref["mi"]).max())
    print(f"[mi-error] {A.shape}x{B.shape} K={KA},{KB} prec={prec} max|dMI|={err:.3e} residual={g['status'][1]:.3e}")
    assert err <= MI_TOL, err
    # gamma-gated peak of Alg. 1: identical, or a near-tie within the MI tolerance
    idx, best, _ = oracle.gamma_argmax(ref["mi"], ref["n"], gamma)
    _, dy, dx, n, mi = g["peak"]
    r, c = dy + A.shape[0] - 1, dx + A.shape[1] - 1
    assert (r * ref["mi"].shape[1] + c == idx) or abs(ref["mi"][r, c] - best) <= MI_TOL
    assert ref["n"][r, c] >= gamma * ref["n"].max()
    return g, ref


def _rand(rng, HA, WA, HB, WB, KA, KB, p0=0.2):
    A = rng.integers(0, KA, (HA, WA)).astype(np.int32)
    B = rng.integers(0, KB, (HB, WB)).astype(np.int32)
    MA = (rng.random((HA, WA)) >= p0).astype(np.uint8)
    MB = (rng.random((HB, WB)) >= p0).astype(np.uint8)
    A[MA == 0] = 999   # ignored under mask 0
    B[MB == 0] = -7
    return A, MA, B, MB


RAGGED = [(1, 1, 1, 1, 1, 1), (1, 5, 3, 1, 2, 3), (7, 9, 5, 6, 5, 4), (17, 33, 20, 11, 3, 7),
          (64, 70, 31, 45, 13, 24), (70, 70, 70, 70, 8, 8), (5, 130, 9, 120, 4, 4)]


@pytest.mark.parametrize("prec_name", ["FP32", "SPLIT32", "FP64"])
@pytest.mark.parametrize("shape", RAGGED, ids=lambda s: "x".join(map(str, s)))
def test_ragged_random(cm, prec_name, shape):
    rng = np.random.default_rng(hash(shape) % 2**32)
    A, MA, B, MB = _rand(rng, *shape)
    check_exact(cm, A, MA, B, MB, shape[4], shape[5], getattr(cm, prec_name), gamma=0.3)


# Wide maps (Q = 1024 / 2048) run the row kernel that keeps the B-marginals in
# Tensor Memory and prefetches Y rows with TMA: K_B = 16 takes its fast path,
# other K_B the general one.  Also check it against the shared-memory kernel.
# Row widths C = W_A + W_B - 1 whose transform width Q is 512, 1024 or 2048 (the
# smallest 2^k or 3 * 2^k >= C), the widths of the Tensor-Memory row kernel.
WIDE = [((20, 450, 30, 500), (16, 16)), ((16, 300, 12, 480), (5, 7)), ((20, 200, 30, 250), (16, 16)),
        ((9, 900, 11, 800), (16, 16)), ((12, 880, 10, 900), (24, 3)), ((16, 240, 12, 260), (5, 7))]


def _transform_width(c):
    return min(n for n in [1 << k for k in range(4, 13)] + [3 << k for k in range(5, 11)] if n >= max(16, c))


@pytest.mark.parametrize("shape,K", WIDE, ids=lambda x: "x".join(map(str, x)))
def test_wide_rows_tmem_path(cm, shape, K, monkeypatch):
    """Q = 512, 1024 and 2048 with no count maps requested run the Tensor-Memory row
    kernel (TMA-staged rows, B-marginals in TMEM; at Q = 1024 the load-once radix-2
    step, at Q = 512 radix-4 teams and one pass per row): N and MI against the
    oracle over the whole map.  The generic kernel
    (CMIF_DISABLE_TMEM=1, with count maps, every count against the oracle) gives
    the same N and bit-identical MI."""
    HA, WA, HB, WB = shape
    assert _transform_width(WA + WB - 1) in (512, 1024, 2048)
    rng = np.random.default_rng(sum(shape) * 7 + K[0])
    A, MA, B, MB = _rand(rng, *shape, *K)
    g = run_gpu(cm, A, MA, B, MB, K[0], K[1], cm.FP32, counts=False, gamma=0.5)
    assert g["status"][0] == "OK" and g["status"][1] < 0.25, g["status"]
    ref = oracle.cmif(A, MA, B, MB, K[0], K[1])
    np.testing.assert_array_equal(g["n"], ref["n"])
    assert float(np.abs(g["mi"] - ref["mi"]).max()) <= MI_TOL
    monkeypatch.setenv("CMIF_DISABLE_TMEM", "1")
    g2, _ = check_exact(cm, A, MA, B, MB, K[0], K[1], cm.FP32, gamma=0.5)
    assert np.array_equal(g2["n"], g["n"]) and np.array_equal(g2["mi"], g["mi"])


@pytest.mark.parametrize("shape,K", WIDE[:3], ids=lambda x: "x".join(map(str, x)))
def test_wide_rows_tmem_auto(cm, shape, K, monkeypatch):
    """CMIF_AUTO at the Tensor-Memory widths: the row kernel's AUTO form (exact
    counts of listed pairs, per-pair residuals) with every pair listed and with the
    default predicate; N and MI against the oracle over the whole map."""
    rng = np.random.default_rng(sum(shape) * 11 + K[1])
    A, MA, B, MB = _rand(rng, *shape, *K)
    ref = oracle.cmif(A, MA, B, MB, K[0], K[1])
    for mode in ("all", None):
        if mode:
            monkeypatch.setenv("CMIF_AUTO_PREDICATE", mode)
        else:
            monkeypatch.delenv("CMIF_AUTO_PREDICATE", raising=False)
        g = run_gpu(cm, A, MA, B, MB, K[0], K[1], cm.AUTO, counts=False, gamma=0.5)
        assert g["status"][0] == "OK" and g["status"][1] < 0.25, (mode, g["status"])
        np.testing.assert_array_equal(g["n"], ref["n"])
        assert float(np.abs(g["mi"] - ref["mi"]).max()) <= MI_TOL


def test_null_masks_and_voronoi(cm):
    rng = np.random.default_rng(11)
    A = synth.make_field(rng, 48, 40, 30, 6).image(48, 40)
    B = synth.make_field(rng, 33, 52, 30, 5).image(33, 52)
    check_exact(cm, A, None, B, None, 6, 5, cm.FP32, gamma=0.5)


def test_empty_mask_gives_zero(cm):
    rng = np.random.default_rng(12)
    A, MA, B, MB = _rand(rng, 20, 20, 20, 20, 4, 4)
    MB[:] = 0
    g = run_gpu(cm, A, MA, B, MB, 4, 4, cm.FP32)
    assert np.all(g["n"] == 0) and np.all(g["mi"] == 0.0)
    assert np.all(g["counts"] == 0)


def test_single_label_is_zero(cm):
    rng = np.random.default_rng(13)
    A = np.zeros((30, 25), np.int32)
    B = np.zeros((22, 31), np.int32)
    MB = (rng.random((22, 31)) > 0.5).astype(np.uint8)
    g, ref = check_exact(cm, A, None, B, MB, 1, 1, cm.FP32)
    assert np.all(g["mi"] == 0.0)


def test_label_range_reported(cm):
    A = np.zeros((16, 16), np.int32)
    A[3, 4] = 5
    B = np.zeros((16, 16), np.int32)
    g = run_gpu(cm, A, None, B, None, 4, 4, cm.FP32, counts=False)
    assert g["status"][0] == "LABEL_RANGE"
    MA = np.ones((16, 16), np.uint8)
    MA[3, 4] = 0
    g = run_gpu(cm, A, MA, B, None, 4, 4, cm.FP32, counts=False)
    assert g["status"][0] == "OK"


@pytest.mark.parametrize("prec_name", ["FP64", "SPLIT32", "FP32"])
def test_plain64_full(cm, prec_name):
    cfg = synth.make_workload("plain-64x64-K8")
    g, ref = check_exact(cm, cfg["A"], cfg["M_A"], cfg["B"], cfg["M_B"], 8, 8, getattr(cm, prec_name), gamma=0.5)
    _, dy, dx, _, _ = g["peak"]
    assert (dy, dx) == tuple(cfg["shift"])


def test_single256_full(cm):
    cfg = synth.make_workload("single-256x256-K16")
    g, ref = check_exact(cm, cfg["A"], cfg["M_A"], cfg["B"], cfg["M_B"], 16, 16, cm.FP32, gamma=0.5)
    _, dy, dx, _, _ = g["peak"]
    assert (dy, dx) == tuple(cfg["shift"])


def _sample_shifts(rng, HA, WA, HB, WB, n, extra=()):
    dys = list(rng.integers(-(HA - 1), HB, n))
    dxs = list(rng.integers(-(WA - 1), WB, n))
    for dy, dx in [(0, 0), (-(HA - 1), -(WA - 1)), (HB - 1, WB - 1), (-(HA - 1), WB - 1), (HB - 1, -(WA - 1)),
                   (1, -1), (-2, 3), *extra]:
        dys.append(dy)
        dxs.append(dx)
    return np.array(dys, np.int32), np.array(dxs, np.int32)


def test_single1024_full_size_sampled(cm):
    """1024^2, K=16, FP32 path at the benchmark size: N exact on the whole map
    (closed form for all-ones masks), MI on sampled shifts vs the oracle,
    residual under the guard, planted shift found."""
    cfg = synth.make_workload("single-1024x1024-K16")
    A, B = cfg["A"], cfg["B"]
    g = run_gpu(cm, A, cfg["M_A"], B, cfg["M_B"], 16, 16, cm.FP32, counts=False, gamma=0.5)
    assert g["status"][0] == "OK" and g["status"][1] < 0.25, g["status"]
    H = 1024
    d = np.arange(2 * H - 1) - (H - 1)
    np.testing.assert_array_equal(g["n"], np.outer(H - np.abs(d), H - np.abs(d)))
    rng = np.random.default_rng(3)
    dys, dxs = _sample_shifts(rng, H, H, H, H, 160, extra=[tuple(cfg["shift"])])
    ref = oracle.cmif_at(A, cfg["M_A"], B, cfg["M_B"], 16, 16, dys, dxs)
    got = g["mi"][dys + H - 1, dxs + H - 1]
    np.testing.assert_array_equal(g["n"][dys + H - 1, dxs + H - 1], ref["n"])
    err = float(np.abs(got - ref["mi"]).max())
    print(f"[mi-error] 1024^2 K=16 sampled max|dMI|={err:.3e} residual={g['status'][1]:.3e}")
    assert err <= MI_TOL, err
    _, dy, dx, _, _ = g["peak"]
    assert (dy, dx) == tuple(cfg["shift"])


def _timed(cm, plan, A, B, mi, n, reps=3):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plan.compute(A, None, B, None, mi, n, None, 0.5)
    ev0.record()
    for _ in range(reps):
        plan.compute(A, None, B, None, mi, n, None, 0.5)
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / reps


@pytest.mark.parametrize("mode", ["predicate", "guard", "guard-fp64"])
def test_auto_per_pair_precision_unbalanced_labels(cm, mode, monkeypatch):
    """A dominant label (98% of 1024^2 pixels) makes the FP32 correlation of the
    pair (0, 0) inexact.  CMIF_AUTO computes that pair in the second precision:
    chosen up front by the predicate, or, with the predicate off, after the FP32
    guard breached (two-term FP32, or FP64 on request).  Only the listed pairs pay
    for it: N exact and MI within tolerance at sampled shifts, and the AUTO map
    costs the FP32 map plus well under the second-precision map it replaced (one
    pair of four listed: about a quarter of it)."""
    if mode != "predicate":
        monkeypatch.setenv("CMIF_AUTO_PREDICATE", "0")
    if mode == "guard-fp64":
        monkeypatch.setenv("CMIF_AUTO_TIER2", "fp64")
    rng = np.random.default_rng(21)
    H = 1024
    A = (rng.random((H, H)) < 0.02).astype(np.int32)
    B = (rng.random((H, H)) < 0.02).astype(np.int32)
    dA, dB = _to(A), _to(B)
    R = 2 * H - 1
    mi = torch.empty((R, R), dtype=torch.float64, device="cuda:0")
    n = torch.empty((R, R), dtype=torch.int32, device="cuda:0")
    p32 = cm.Plan(H, H, H, H, 2, 2, cm.FP32)
    pa = cm.Plan(H, H, H, H, 2, 2, cm.AUTO)
    t32 = _timed(cm, p32, dA, dB, mi, n)
    st32 = p32.status()
    p2 = cm.Plan(H, H, H, H, 2, 2, cm.FP64 if mode == "guard-fp64" else cm.SPLIT32)
    t2 = _timed(cm, p2, dA, dB, mi, n)
    p2.close()
    assert st32[0] == "PRECISION" and st32[1] >= 0.25, st32     # FP32 alone is not exact here
    ta = _timed(cm, pa, dA, dB, mi, n)
    st = pa.status()
    pred, esc, r32, r2 = pa.precision_report()
    print(f"[auto-{mode}] FP32 {t32:.2f} ms (residual {st32[1]:.3f}), whole map in the second precision "
          f"{t2:.2f} ms, AUTO {ta:.2f} ms: {pred} predicted, "
          f"{esc} escalated, residual FP32 pairs {r32:.3e}, second precision {r2:.3e}")
    assert st[0] == "OK" and st[1] < 0.25, st
    assert r32 < 0.25 and r2 < 0.25
    if mode == "predicate":
        assert pred >= 1 and esc == 0
    else:
        assert pred == 0 and esc >= 1
    assert pred + esc < 4                                        # not every pair: the small labels stay FP32
    pa.set_profiling(True)
    pa.compute(dA, None, dB, None, mi, n, None, 0.5)
    print(f"[auto-{mode}] launches: " + ", ".join(f"{k} {v:.3f}" for k, v in pa.stage_times()))
    pa.set_profiling(False)
    assert ta < t32 + 0.6 * t2, (ta, t32, t2)
    dys, dxs = _sample_shifts(rng, H, H, H, H, 64)
    ref = oracle.cmif_at(A, None, B, None, 2, 2, dys, dxs)
    got_mi, got_n = mi.cpu().numpy(), n.cpu().numpy()
    np.testing.assert_array_equal(got_n[dys + H - 1, dxs + H - 1], ref["n"])
    assert float(np.abs(got_mi[dys + H - 1, dxs + H - 1] - ref["mi"]).max()) <= MI_TOL
    p32.close()
    pa.close()


@pytest.mark.parametrize("shape", RAGGED[2:], ids=lambda s: "x".join(map(str, s)))
def test_auto_every_pair_listed_exact(cm, shape, monkeypatch):
    """CMIF_AUTO with every pair sent to the second precision up front
    (CMIF_AUTO_PREDICATE=all; pairs beyond the 128-slot list keep FP32): the FP32
    row pass takes the listed pairs' counts from the second precision, and every
    count (joint, marginals, N) still matches the oracle exactly."""
    monkeypatch.setenv("CMIF_AUTO_PREDICATE", "all")
    rng = np.random.default_rng(sum(shape) + 5)
    A, MA, B, MB = _rand(rng, *shape)
    check_exact(cm, A, MA, B, MB, shape[4], shape[5], cm.AUTO, gamma=0.4)


def test_host_buffer_entry_point(cm):
    cfg = synth.make_workload("plain-64x64-K8")
    A, B = cfg["A"], cfg["B"]
    plan = cm.Plan(64, 64, 64, 64, 8, 8, cm.FP32)
    mi = np.empty((127, 127), np.float64)
    n = np.empty((127, 127), np.int32)
    pk = cm.Peak()
    plan.compute_host(A, cfg["M_A"], B, cfg["M_B"], mi, n, 0.5, pk)
    ref = oracle.cmif(A, cfg["M_A"], B, cfg["M_B"], 8, 8)
    np.testing.assert_array_equal(n, ref["n"])
    assert float(np.abs(mi - ref["mi"]).max()) <= MI_TOL
    assert (pk.dy, pk.dx) == tuple(cfg["shift"])
    plan.close()


@pytest.mark.parametrize("shape,K,prec", [((40, 70, 50, 60), 5, "FP32"), ((100, 300, 90, 260), 6, "FP32"),
                                          ((33, 41, 29, 37), 4, "FP64")])
def test_host_entry_pinned_outputs(cm, shape, K, prec):
    """Output maps in pinned host memory are written by the kernels directly (no copy
    after the map), pageable ones by a copy: both equal the oracle (N exactly, MI within
    the tolerance) and each other bit for bit, and so does the peak."""
    rng = np.random.default_rng(sum(shape) + K)
    A, MA, B, MB = _rand(rng, *shape, K, K)
    HA, WA, HB, WB = shape
    R, C = HA + HB - 1, WA + WB - 1
    ref = oracle.cmif(A, MA, B, MB, K, K)
    plan = cm.Plan(*shape, K, K, getattr(cm, prec))
    mi_p = torch.full((R, C), float("nan"), dtype=torch.float64).pin_memory()
    n_p = torch.full((R, C), -1, dtype=torch.int32).pin_memory()
    pk_p = cm.Peak()
    plan.compute_host(A, MA, B, MB, mi_p, n_p, 0.5, pk_p)
    mi_h = np.full((R, C), np.nan)
    n_h = np.full((R, C), -1, np.int32)
    pk_h = cm.Peak()
    plan.compute_host(A, MA, B, MB, mi_h, n_h, 0.5, pk_h)
    assert plan.status()[0] == "OK"
    plan.close()
    np.testing.assert_array_equal(n_p.numpy(), ref["n"])
    assert float(np.abs(mi_p.numpy() - ref["mi"]).max()) <= MI_TOL
    assert np.array_equal(mi_p.numpy(), mi_h) and np.array_equal(n_p.numpy(), n_h)
    assert (pk_p.dy, pk_p.dx, pk_p.n, pk_p.mi) == (pk_h.dy, pk_h.dx, pk_h.n, pk_h.mi)


def test_max_label_count_exact(cm):
    """K_A = K_B = 64 (the largest accepted): 4096 label pairs; exact counts on the
    whole map, FP32 and FP64."""
    rng = np.random.default_rng(64)
    A, MA, B, MB = _rand(rng, 23, 31, 19, 27, 64, 64, p0=0.1)
    for prec in (cm.FP32, cm.FP64):
        check_exact(cm, A, MA, B, MB, 64, 64, prec, gamma=0.3)


def test_max_k_wide_rows_global_b_marginals(cm):
    """K_B = 64 at Q = 2048: the B-marginals (64 x 2048 floats) fit neither TMEM
    nor shared memory, so the row kernel keeps them in its global slice."""
    rng = np.random.default_rng(65)
    A, MA, B, MB = _rand(rng, 9, 600, 7, 610, 5, 64, p0=0.05)
    g = run_gpu(cm, A, MA, B, MB, 5, 64, cm.FP32, counts=False, gamma=0.2)
    ref = oracle.cmif(A, MA, B, MB, 5, 64)
    assert g["status"][0] == "OK", g["status"]
    np.testing.assert_array_equal(g["n"], ref["n"])
    assert float(np.abs(g["mi"] - ref["mi"]).max()) <= MI_TOL


@pytest.mark.parametrize("KA,KB", [(3, 17), (5, 24)])
def test_wide_3x_rows_global_b_marginals(cm, KA, KB):
    """Q = 3072 rows (output width 2299) with the B-marginals in the row kernel's
    global slice (K_B x 3072 floats do not fit in shared memory): every round of
    four pairs loads its slots together.  K_B = 17: A's label changes inside
    rounds and the last round is shorter (one pair at a time); K_B = 24: whole
    rounds throughout."""
    rng = np.random.default_rng(68 + KB)
    A, MA, B, MB = _rand(rng, 4, 1100, 5, 1200, KA, KB, p0=0.05)
    g = run_gpu(cm, A, MA, B, MB, KA, KB, cm.FP32, counts=False, gamma=0.2)
    ref = oracle.cmif(A, MA, B, MB, KA, KB)
    assert g["status"][0] == "OK", g["status"]
    np.testing.assert_array_equal(g["n"], ref["n"])
    assert float(np.abs(g["mi"] - ref["mi"]).max()) <= MI_TOL


def test_extreme_aspect_max_row_transform(cm):
    """1 x 2048 rows: P = 16 (the smallest transform), Q = 4096 (the largest)."""
    rng = np.random.default_rng(66)
    A, MA, B, MB = _rand(rng, 1, 2048, 1, 2048, 3, 3, p0=0.1)
    check_exact(cm, A, MA, B, MB, 3, 3, cm.FP32, gamma=0.5)


def test_max_transform_size_sampled(cm):
    """2048^2 pair (the largest plan: P = Q = 4096), K = 4, AUTO precision: N
    exact on the whole map (all-ones masks: closed form), MI and N at sampled
    shifts vs the oracle, residual guard satisfied after any escalation."""
    rng = np.random.default_rng(67)
    H = 2048
    A = rng.integers(0, 4, (H, H)).astype(np.int32)
    A[: H // 2, : H // 3] = 1
    B = np.roll(A, (37, -101), axis=(0, 1))
    B[rng.random(B.shape) < 0.1] = 2
    g = run_gpu(cm, A, None, B, None, 4, 4, cm.AUTO, counts=False, gamma=0.5)
    assert g["status"][0] == "OK", g["status"]
    d = np.arange(2 * H - 1) - (H - 1)
    np.testing.assert_array_equal(g["n"], np.outer(H - np.abs(d), H - np.abs(d)))
    dys, dxs = _sample_shifts(rng, H, H, H, H, 40, extra=[(37, -101)])
    ref = oracle.cmif_at(A, None, B, None, 4, 4, dys, dxs)
    np.testing.assert_array_equal(g["n"][dys + H - 1, dxs + H - 1], ref["n"])
    err = float(np.abs(g["mi"][dys + H - 1, dxs + H - 1] - ref["mi"]).max())
    print(f"[mi-error] 2048^2 K=4 AUTO sampled max|dMI|={err:.3e} status={g['status']}")
    assert err <= MI_TOL, err
    assert tuple(g["peak"][1:3]) == (37, -101)


# Shapes whose output ranges pick transform lengths 3 * 2^k (96 .. 3072) in FP32 plans:
# (H_A, W_A, H_B, W_B, K_A, K_B) -> P x Q
MIXED = [(40, 50, 41, 47, 5, 6),        # 96 x 96
         (70, 100, 90, 60, 4, 3),       # 192 x 192
         (150, 20, 140, 30, 3, 4),      # 384 x 64
         (8, 300, 9, 400, 5, 5),        # 16 x 768
         (5, 700, 4, 800, 3, 3),        # 16 x 1536
         (3, 1100, 4, 1200, 2, 2),      # 16 x 3072
         (1300, 3, 1200, 2, 2, 3)]      # 3072 x 16


@pytest.mark.parametrize("shape", MIXED, ids=lambda s: "x".join(map(str, s)))
def test_mixed_radix_lengths_exact(cm, shape):
    """FP32 plans take transform lengths 3 * 2^k (radix-3 and radix-6 steps) when
    they are shorter than the next power of two; counts stay bit-exact."""
    rng = np.random.default_rng(sum(shape) * 3)
    A, MA, B, MB = _rand(rng, *shape)
    check_exact(cm, A, MA, B, MB, shape[4], shape[5], cm.FP32, gamma=0.3)


def test_mixed_radix_equals_power_of_two(cm, monkeypatch):
    """A 768^2 pair (output range 1535: length 1536 instead of 2048): the same N and
    MI as the power-of-two plan, bit for bit (MI comes from exact integer sums),
    and the oracle's values at sampled shifts."""
    rng = np.random.default_rng(768)
    H, K = 768, 8
    A, B = synth.planted_pair(rng, H, H, 900, K, K, (31, -17), 0.1, same_labels=True)
    monkeypatch.setenv("CMIF_ROWS_POW2", "0")  # rows of width 1536 too, not only the columns
    outs = []
    for pow2 in (False, True):
        if pow2:
            monkeypatch.setenv("CMIF_POW2_ONLY", "1")
        g = run_gpu(cm, A, None, B, None, K, K, cm.FP32, counts=False, gamma=0.5)
        assert g["status"][0] == "OK", g["status"]
        outs.append(g)
    assert np.array_equal(outs[0]["n"], outs[1]["n"]) and np.array_equal(outs[0]["mi"], outs[1]["mi"])
    dys, dxs = _sample_shifts(rng, H, H, H, H, 48, extra=[(31, -17)])
    ref = oracle.cmif_at(A, None, B, None, K, K, dys, dxs)
    np.testing.assert_array_equal(outs[0]["n"][dys + H - 1, dxs + H - 1], ref["n"])
    assert float(np.abs(outs[0]["mi"][dys + H - 1, dxs + H - 1] - ref["mi"]).max()) <= MI_TOL
