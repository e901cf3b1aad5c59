"""Pins for the CPU oracle against things other than itself.

* hand-derived values (tests/golden/hand_cases.txt),
* scikit-learn's mutual_info_score on the explicitly cut-out overlap,
* brute force through Eq. mi (the p log p/(p p) form) instead of the
  entropy form Eq. mientropy that the oracle uses,
* closed forms (N for full masks, MI(0) = H(A) for A = B, K = 1 => 0),
* invariants (marginals = sums of joints = bincounts of the overlap,
  label-permutation invariance, the swap symmetry, 0 <= MI <= min(H_A, H_B)),
* the planted shift of the synthetic workloads,
* mutation tests: a plausible mistake planted in a copy of the oracle's C
  source must make one of these pins fail.
"""
import math
import os
import re
import subprocess
import tempfile
import ctypes

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.txt")


def _parse_golden():
    cases, cur = [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, _, rest = line.partition(" ")
        if key == "case":
            cur = {"name": rest}
            cases.append(cur)
        elif key in ("A", "MA", "B", "MB"):
            shape, _, vals = rest.partition(":")
            h, w = map(int, shape.split())
            cur[key] = np.array([int(v) for v in vals.split()]).reshape(h, w)
        elif key == "K":
            cur["K"] = tuple(map(int, rest.split()))
        else:
            cur[key] = np.array([float(v) for v in rest.split()])
    return cases


@pytest.mark.parametrize("case", _parse_golden(), ids=lambda c: c["name"])
def test_hand_cases(case):
    out = oracle.cmif(case["A"], case["MA"], case["B"], case["MB"], *case["K"])
    assert np.array_equal(out["n"].ravel(), case["N"].astype(np.int64))
    np.testing.assert_allclose(out["mi"].ravel(), case["MI"], atol=1e-15, rtol=0)


def _overlap(A, MA, B, MB, dy, dx):
    """Cut the overlap of A and the shifted B out explicitly (numpy slicing)."""
    HA, WA = A.shape
    HB, WB = B.shape
    y0, y1 = max(0, -dy), min(HA, HB - dy)
    x0, x1 = max(0, -dx), min(WA, WB - dx)
    a = A[y0:y1, x0:x1]
    b = B[y0 + dy:y1 + dy, x0 + dx:x1 + dx]
    m = MA[y0:y1, x0:x1].astype(bool) & MB[y0 + dy:y1 + dy, x0 + dx:x1 + dx].astype(bool)
    return a[m], b[m]


def _random_case(rng, HA, WA, HB, WB, KA, KB, p_mask=0.2):
    A = rng.integers(0, KA, (HA, WA)).astype(np.int32)
    B = rng.integers(0, KB, (HB, WB)).astype(np.int32)
    MA = (rng.random((HA, WA)) >= p_mask).astype(np.uint8)
    MB = (rng.random((HB, WB)) >= p_mask).astype(np.uint8)
    # labels under mask 0 may be anything
    A[MA == 0] = rng.integers(-5, 100, int((MA == 0).sum()))
    B[MB == 0] = rng.integers(-5, 100, int((MB == 0).sum()))
    return A, MA, B, MB


def test_against_sklearn_mutual_info():
    metrics = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(1)
    for (HA, WA, HB, WB, KA, KB) in [(7, 9, 5, 6, 3, 4), (12, 10, 12, 10, 5, 5), (4, 13, 9, 3, 2, 7)]:
        A, MA, B, MB = _random_case(rng, HA, WA, HB, WB, KA, KB)
        out = oracle.cmif(A, MA, B, MB, KA, KB)
        for r in range(HA + HB - 1):
            for c in range(WA + WB - 1):
                dy, dx = r - (HA - 1), c - (WA - 1)
                a, b = _overlap(A, MA, B, MB, dy, dx)
                assert out["n"][r, c] == a.size
                ref = metrics.mutual_info_score(a, b) / math.log(2) if a.size else 0.0
                assert abs(out["mi"][r, c] - ref) < 1e-12, (dy, dx)


def _mi_eq_mi(a, b):
    """Eq. mi written as a plain double loop over histogram bins (not the entropy form)."""
    n = len(a)
    if n == 0:
        return 0.0
    joint, pa, pb = {}, {}, {}
    for u, v in zip(a.tolist(), b.tolist()):
        joint[(u, v)] = joint.get((u, v), 0) + 1
        pa[u] = pa.get(u, 0) + 1
        pb[v] = pb.get(v, 0) + 1
    s = 0.0
    for (u, v), c in joint.items():
        p = c / n
        s += p * math.log2(p / ((pa[u] / n) * (pb[v] / n)))
    return s


def test_brute_force_eq_mi_and_marginals():
    rng = np.random.default_rng(2)
    HA, WA, HB, WB, KA, KB = 6, 8, 9, 5, 4, 3
    A, MA, B, MB = _random_case(rng, HA, WA, HB, WB, KA, KB)
    out = oracle.cmif(A, MA, B, MB, KA, KB, counts=True, marginals=True, entropies=True)
    for r in range(HA + HB - 1):
        for c in range(WA + WB - 1):
            dy, dx = r - (HA - 1), c - (WA - 1)
            a, b = _overlap(A, MA, B, MB, dy, dx)
            assert abs(out["mi"][r, c] - _mi_eq_mi(a, b)) < 1e-12
            J = out["joint"][:, r, c].reshape(KA, KB)
            ref = np.zeros((KA, KB), np.int64)
            np.add.at(ref, (a, b), 1)
            assert np.array_equal(J, ref)
            assert np.array_equal(out["marg_a"][:, r, c], np.bincount(a, minlength=KA))
            assert np.array_equal(out["marg_b"][:, r, c], np.bincount(b, minlength=KB))
            assert J.sum() == out["n"][r, c]
            assert np.array_equal(J.sum(axis=1), out["marg_a"][:, r, c])
            assert np.array_equal(J.sum(axis=0), out["marg_b"][:, r, c])


def test_n_closed_form_full_masks():
    rng = np.random.default_rng(3)
    for (HA, WA, HB, WB) in [(9, 7, 9, 7), (5, 11, 8, 3)]:
        A = rng.integers(0, 3, (HA, WA))
        B = rng.integers(0, 3, (HB, WB))
        out = oracle.cmif(A, None, B, None, 3, 3)
        dy = np.arange(HA + HB - 1) - (HA - 1)
        dx = np.arange(WA + WB - 1) - (WA - 1)
        ny = np.minimum(HA, HB - dy) - np.maximum(0, -dy)
        nx = np.minimum(WA, WB - dx) - np.maximum(0, -dx)
        assert np.array_equal(out["n"], np.outer(ny, nx))
        if HA == HB and WA == WB:
            assert np.array_equal(out["n"], np.outer(HA - abs(dy), WA - abs(dx)))


def test_self_alignment_is_label_entropy():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(4)
    A = synth.make_field(rng, 40, 33, 25, 6).image(40, 33)
    out = oracle.cmif(A, None, A, None, 6, 6, entropies=True)
    hist = np.bincount(A.ravel(), minlength=6)
    h = stats.entropy(hist, base=2)
    r0, c0 = 39, 32
    assert abs(out["mi"][r0, c0] - h) < 1e-12
    assert abs(out["ent"][0, r0, c0] - h) < 1e-12
    assert int(np.argmax(out["mi"])) != -1


def test_k1_is_zero_and_bounds():
    rng = np.random.default_rng(5)
    A = np.zeros((6, 7), np.int32)
    B = np.zeros((5, 9), np.int32)
    out = oracle.cmif(A, None, B, None, 1, 1)
    assert np.all(out["mi"] == 0.0)
    A, MA, B, MB = _random_case(rng, 8, 8, 7, 9, 4, 5)
    out = oracle.cmif(A, MA, B, MB, 4, 5, entropies=True)
    hA, hB = out["ent"][0], out["ent"][1]
    assert np.all(out["mi"] >= -1e-12)
    assert np.all(out["mi"] <= np.minimum(hA, hB) + 1e-12)


def test_permutation_and_swap_symmetry():
    rng = np.random.default_rng(6)
    A, MA, B, MB = _random_case(rng, 9, 6, 7, 8, 5, 4)
    base = oracle.cmif(A, MA, B, MB, 5, 4)
    perm = rng.permutation(4)
    Bp = np.where(MB == 1, perm[np.clip(B, 0, 3)], B)
    permd = oracle.cmif(A, MA, Bp, MB, 5, 4)
    np.testing.assert_allclose(permd["mi"], base["mi"], atol=1e-12, rtol=0)
    swapped = oracle.cmif(B, MB, A, MA, 4, 5)
    np.testing.assert_allclose(swapped["mi"][::-1, ::-1], base["mi"], atol=1e-12, rtol=0)
    assert np.array_equal(swapped["n"][::-1, ::-1], base["n"])


def test_cmif_at_matches_full_map():
    rng = np.random.default_rng(7)
    A, MA, B, MB = _random_case(rng, 10, 12, 11, 7, 4, 6)
    full = oracle.cmif(A, MA, B, MB, 4, 6, counts=True)
    dys = rng.integers(-9, 11, 40)
    dxs = rng.integers(-11, 7, 40)
    at = oracle.cmif_at(A, MA, B, MB, 4, 6, dys, dxs, counts=True)
    r, c = dys + 9, dxs + 11
    assert np.array_equal(at["mi"], full["mi"][r, c])
    assert np.array_equal(at["n"], full["n"][r, c])
    assert np.array_equal(at["joint"], full["joint"][:, r, c].T)


def test_label_range_rejected():
    A = np.array([[0, 1], [2, 0]], np.int32)
    with pytest.raises(oracle.OracleError):
        oracle.cmif(A, None, A, None, 2, 3)
    MA = np.array([[1, 1], [0, 1]], np.uint8)      # the bad label sits under mask 0
    oracle.cmif(A, MA, A, None, 2, 3)


def test_planted_shift_recovered():
    cfg = synth.make_workload("plain-64x64-K8")
    out = oracle.cmif(cfg["A"], cfg["M_A"], cfg["B"], cfg["M_B"], cfg["K_A"], cfg["K_B"])
    idx, mi, n = oracle.gamma_argmax(out["mi"], out["n"], 0.5)
    r, c = divmod(idx, out["mi"].shape[1])
    assert (r - 63, c - 63) == tuple(cfg["shift"])
    cfg = synth.make_workload("single-256x256-K16", scale=0.25)
    out = oracle.cmif(cfg["A"], cfg["M_A"], cfg["B"], cfg["M_B"], cfg["K_A"], cfg["K_B"])
    idx, mi, n = oracle.gamma_argmax(out["mi"], out["n"], 0.5)
    H = cfg["A"].shape[0]
    r, c = divmod(idx, out["mi"].shape[1])
    assert (r - (H - 1), c - (H - 1)) == tuple(cfg["shift"])


def test_gamma_argmax_and_align_rules():
    mi = np.array([[0.1, 0.9, 0.5], [0.9, 0.2, 0.95]])
    n = np.array([[10, 2, 10], [10, 10, 4]])
    # gamma 0: the global max 0.95
    assert oracle.gamma_argmax(mi, n, 0.0)[0] == 5
    # gamma 0.5: N >= 5 excludes index 1 (N=2) and index 5 (N=4); tie 0.9 at 1 is excluded,
    # the lowest index among the remaining maxima (0.9 at index 3) wins
    assert oracle.gamma_argmax(mi, n, 0.5)[0] == 3
    # gamma 1: N >= max N (Alg. 1's gate is inclusive) keeps only the maximal overlaps;
    # for full masks of equal size that is chi = 0 alone, whatever the MI elsewhere
    rng = np.random.default_rng(6)
    A = rng.integers(0, 3, (7, 9)).astype(np.int32)
    B = rng.integers(0, 3, (7, 9)).astype(np.int32)
    ref = oracle.cmif(A, None, B, None, 3, 3)
    idx, _, n0 = oracle.gamma_argmax(ref["mi"], ref["n"], 1.0)
    assert divmod(idx, 17) == (6, 8) and n0 == 63
    maps = [(mi, n), (mi * 0 + 0.9, n), (mi + 0.5, n)]
    best, top = oracle.align(maps, 0.5, top_k=3)
    assert best[0] == 2 and abs(best[2] - 1.4) < 1e-15
    # equal I_T: the earlier transform stays (strict >); top-k keeps angle order for ties
    best, top = oracle.align([(mi, n), (mi, n)], 0.5, top_k=2)
    assert best[0] == 0 and [t[0] for t in top] == [0, 1]
    # nothing beats I = 0: T-hat stays the identity
    best, _ = oracle.align([(np.zeros((2, 2)), np.ones((2, 2), int))], 0.0)
    assert best[0] == -1


def test_warp_identity_and_quarter_turn():
    rng = np.random.default_rng(8)
    for H in (7, 8):
        B = rng.integers(0, 9, (H, H)).astype(np.int32)
        M = (rng.random((H, H)) > 0.3).astype(np.uint8)
        oB, oM = oracle.warp_nn(B, M, 0.0)
        assert np.array_equal(oM, M) and np.array_equal(oB[M == 1], B[M == 1])
        oB, oM = oracle.warp_nn(B, None, math.pi / 2)
        assert np.all(oM == 1) and np.array_equal(oB, np.rot90(B, 1))
        oB, oM = oracle.warp_nn(B, M, math.pi)
        assert np.array_equal(oM, np.rot90(M, 2)) and np.array_equal(oB[oM == 1], np.rot90(B, 2)[oM == 1])
    # non-square 45 degrees: centre pixel keeps its label, out-of-support corners are masked
    B = rng.integers(0, 5, (9, 15)).astype(np.int32)
    oB, oM = oracle.warp_nn(B, None, math.pi / 4)
    assert oB[4, 7] == B[4, 7] and oM[0, 0] == 0


# ---------------------------------------------------------------------------
# Mutation tests: plant a plausible mistake in a copy of the oracle source and
# check that the pins above notice it.

_MUTATIONS = {
    "drop_last_joint_term": ("HAB += neg_plogp(J[(size_t)a * KB + b], N);",
                             "if (a * KB + b != KA * KB - 1) HAB += neg_plogp(J[(size_t)a * KB + b], N);"),
    "wrong_shift_sign": ("const int32_t *br = B + (size_t)(y + dy) * WB + dx;",
                         "const int32_t *br = B + (size_t)(y + dy) * WB - dx;"),
    "x_range_off_by_one": ("int x0 = dx < 0 ? -dx : 0,", "int x0 = dx < 0 ? -dx + 1 : 0,"),
    "natural_log": ("return -p * log2(p);", "return -p * log(p);"),
    "ignore_mask_b": ("if (mbr && !mbr[x]) continue;", ""),
}


def _build_mutant(name):
    src = open(oracle._SRC).read()
    old, new = _MUTATIONS[name]
    assert old in src
    src = src.replace(old, new)
    d = tempfile.mkdtemp(prefix="oracle_mut_")
    cpath, so = os.path.join(d, "m.c"), os.path.join(d, "m.so")
    open(cpath, "w").write(src)
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", cpath, "-o", so, "-lm"])
    return so


_RUN_PINS = r"""
import ctypes, sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import oracle, test_oracle as t
mut = ctypes.CDLL({so!r})
P, I = ctypes.c_void_p, ctypes.c_int
mut.oracle_cmif.argtypes = [P, P, I, I, P, P, I, I, I, I, P, P, P, P, P, P, I]
mut.oracle_cmif_at.argtypes = [P, P, I, I, P, P, I, I, I, I, I, P, P, P, P, P, P, I]
mut.oracle_warp_nn.argtypes = [P, P, I, I, ctypes.c_double, P, P]
oracle._lib = mut
pins = [lambda: [t.test_hand_cases(c) for c in t._parse_golden()],
        t.test_against_sklearn_mutual_info, t.test_brute_force_eq_mi_and_marginals,
        t.test_n_closed_form_full_masks, t.test_self_alignment_is_label_entropy]
failed = 0
for pin in pins:
    try:
        pin()
    except (AssertionError, oracle.OracleError):
        failed += 1
sys.exit(3 if failed else 0)
"""


@pytest.mark.parametrize("name", sorted(_MUTATIONS))
def test_mutants_are_caught(name):
    """Each mutant runs in a child process (a planted index bug may crash it);
    any pin failure, or a crash, counts as caught."""
    import sys
    so = _build_mutant(name)
    here = os.path.dirname(os.path.abspath(__file__))
    code = _RUN_PINS.format(root=os.path.dirname(here), tests=here, so=so)
    rc = subprocess.run([sys.executable, "-c", code], capture_output=True, timeout=300).returncode
    assert rc != 0, f"mutation {name} was not caught by any pin"
