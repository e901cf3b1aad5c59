"""CPU oracle for the CMIF: the paper's direct histogram method (Sec. 2.2).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library ``paper_2106_14699_gb300``
and neither imports the other; the only common module is ``synth`` (input
generators, which hold none of the method's arithmetic).

Functions and the passages they follow:

* ``cmif``        -- the full CMIF map by the direct method (Sec. 2.2), entropies
                     per Eq. margentropy / Eq. jointentropy on relative frequencies
                     (Eq. finalentropy), MI by Eq. mientropy; 0/0 = 0, 0 log 0 = 0
                     (Sec. 3.2).  Pinned by tests/test_oracle.py.
* ``cmif_at``     -- the same at a list of displacements.  Pinned (same code path).
* ``warp_nn``     -- nearest-neighbour rotation of B (Sec. 3.6); the paper leaves
                     centre, canvas and sign open, the reading is documented in
                     cmif_direct.c.  Pinned by quarter-turn / identity cases.
* ``gamma_argmax``, ``align`` -- the per-transform gamma-gated argmax and the
                     strict-greater update over transforms of Alg. 1.  Pinned by
                     hand-built cases.
* ``alg1_padded`` -- one transform of Alg. 1 with its ZERO-PAD step (Alg. 1,
                     Sec. 3.6): A and M_A padded by ceil(|X_B|_i (1 - gamma))
                     zeros along each axis, the direct CMIF of the padded pair, X_S
                     = the shifts that keep B's domain inside padded A's, and the
                     gated argmax over X_S.  Pinned by tests/test_oracle.py
                     (padding changes nothing inside X_S; full-mask cases).
* ``nmi``         -- the normalised MI the paper cites next to MI (Sec. 2.1),
                     (H_A + H_B) / H_AB from the direct method's entropies, 0/0 = 0.
                     Pinned by closed forms (A = B: 2; independent labels: 1).
* ``swmi``        -- spatially weighted MI (Sec. 3.3): the direct weighted histogram
                     per displacement (each overlapping pixel pair adds W_A W_B to its
                     joint bin), MI by Eq. mi on the weighted relative frequencies.
                     numpy, small inputs.  Pinned by tests/test_oracle_alg1.py (unit
                     weights = MI, 0/1 weights = masked MI, scale invariance, and the
                     weighted label entropy for A = B).
* ``cmif3``       -- the CMIF of two label VOLUMES (Sec. 3.1 with n = 3) by the
                     direct method: at every displacement (dz, dy, dx) the joint
                     histogram of the overlapping voxels, MI by Eq. mi.  numpy, small
                     inputs.  Pinned by tests/test_oracle_alg1.py (depth 1 = the C
                     oracle, N closed form, MI(0) = H(A), swap symmetry).
* ``align_two_stage`` -- the two-stage rigid search of Sec. 3.6 (grid, then random
                     refinement in [theta - 2 pi/|Omega|, theta + 2 pi/|Omega|]), the
                     uniform draws passed in.  Pinned by hand-checked compositions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "liboracle_cmif.so")
_SRC = os.path.join(_HERE, "cmif_direct.c")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_LABEL_RANGE, ERR_INTERNAL = 0, 1, 2, 3


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain C + OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIBPATH) or os.path.getmtime(_LIBPATH) < os.path.getmtime(_SRC):
        tmp = _LIBPATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIBPATH)
            P = ctypes.c_void_p
            I = ctypes.c_int
            lib.oracle_cmif.argtypes = [P, P, I, I, P, P, I, I, I, I, P, P, P, P, P, P, I]
            lib.oracle_cmif.restype = I
            lib.oracle_cmif_at.argtypes = [P, P, I, I, P, P, I, I, I, I, I, P, P, P, P, P, P, I]
            lib.oracle_cmif_at.restype = I
            lib.oracle_warp_nn.argtypes = [P, P, I, I, ctypes.c_double, P, P]
            lib.oracle_warp_nn.restype = I
            lib.oracle_max_threads.argtypes = []
            lib.oracle_max_threads.restype = I
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _prep(A, M_A, B, M_B):
    A = np.ascontiguousarray(A, np.int32)
    B = np.ascontiguousarray(B, np.int32)
    M_A = None if M_A is None else np.ascontiguousarray(M_A, np.uint8)
    M_B = None if M_B is None else np.ascontiguousarray(M_B, np.uint8)
    if A.ndim != 2 or B.ndim != 2:
        raise ValueError("A and B must be 2-D label images")
    if M_A is not None and M_A.shape != A.shape or M_B is not None and M_B.shape != B.shape:
        raise ValueError("mask shape mismatch")
    return A, M_A, B, M_B


def _check(st):
    if st == ERR_LABEL_RANGE:
        raise OracleError("label outside [0, K) under mask")
    if st != OK:
        raise OracleError(f"oracle status {st}")


def cmif(A, M_A, B, M_B, K_A, K_B, *, counts=False, marginals=False, entropies=False, nthreads=0):
    """Full CMIF map over the linear shift range (direct method, Sec. 2.2).

    Returns dict with ``mi`` (R x C float64 bits), ``n`` (R x C int64) and,
    on request, ``joint`` (K_A*K_B x R x C int32), ``marg_a``, ``marg_b``,
    ``ent`` (3 x R x C: H_A, H_B, H_AB).  Row r <-> dy = r - (H_A-1),
    column c <-> dx = c - (W_A-1).
    """
    A, M_A, B, M_B = _prep(A, M_A, B, M_B)
    HA, WA = A.shape
    HB, WB = B.shape
    R, C = HA + HB - 1, WA + WB - 1
    mi = np.empty((R, C), np.float64)
    n = np.empty((R, C), np.int64)
    joint = np.empty((K_A * K_B, R, C), np.int32) if counts else None
    ma = np.empty((K_A, R, C), np.int32) if marginals else None
    mb = np.empty((K_B, R, C), np.int32) if marginals else None
    ent = np.empty((3, R, C), np.float64) if entropies else None
    st = _load().oracle_cmif(_ptr(A), _ptr(M_A), HA, WA, _ptr(B), _ptr(M_B), HB, WB, K_A, K_B,
                             _ptr(mi), _ptr(n), _ptr(joint), _ptr(ma), _ptr(mb), _ptr(ent), nthreads)
    _check(st)
    out = dict(mi=mi, n=n)
    if counts:
        out["joint"] = joint
    if marginals:
        out["marg_a"], out["marg_b"] = ma, mb
    if entropies:
        out["ent"] = ent
    return out


def cmif_at(A, M_A, B, M_B, K_A, K_B, dys, dxs, *, counts=False, entropies=False, nthreads=0):
    """CMIF, N (and optionally joint counts, entropies) at the displacements (dys[i], dxs[i])."""
    A, M_A, B, M_B = _prep(A, M_A, B, M_B)
    HA, WA = A.shape
    HB, WB = B.shape
    dys = np.ascontiguousarray(dys, np.int32)
    dxs = np.ascontiguousarray(dxs, np.int32)
    m = len(dys)
    mi = np.empty(m, np.float64)
    n = np.empty(m, np.int64)
    joint = np.empty((m, K_A * K_B), np.int32) if counts else None
    ent = np.empty((m, 3), np.float64) if entropies else None
    st = _load().oracle_cmif_at(_ptr(A), _ptr(M_A), HA, WA, _ptr(B), _ptr(M_B), HB, WB, K_A, K_B,
                                m, _ptr(dys), _ptr(dxs), _ptr(mi), _ptr(n), _ptr(joint), _ptr(ent), nthreads)
    _check(st)
    out = dict(mi=mi, n=n)
    if counts:
        out["joint"] = joint
    if entropies:
        out["ent"] = ent
    return out


def warp_nn(B, M_B, theta):
    """Nearest-neighbour rotation of (B, M_B) by theta radians (reading in cmif_direct.c)."""
    B = np.ascontiguousarray(B, np.int32)
    M_B = None if M_B is None else np.ascontiguousarray(M_B, np.uint8)
    H, W = B.shape
    oB = np.empty_like(B)
    oM = np.empty((H, W), np.uint8)
    _check(_load().oracle_warp_nn(_ptr(B), _ptr(M_B), H, W, float(theta), _ptr(oB), _ptr(oM)))
    return oB, oM


def gamma_argmax(mi, n, gamma):
    """One transform of Alg. 1: Ncal = gamma * max_chi N; the chi maximising CMIF
    among shifts with N >= Ncal.  Ties go to the lowest row-major map index.
    Returns (flat index, MI there, N there)."""
    mi = np.asarray(mi, np.float64).ravel()
    n = np.asarray(n).ravel()
    thr = float(gamma) * float(n.max()) if n.size else 0.0
    ok = n.astype(np.float64) >= thr
    masked = np.where(ok, mi, -np.inf)
    idx = int(np.argmax(masked))
    return idx, float(mi[idx]), int(n[idx])


def align(per_angle, gamma, top_k=1):
    """Alg. 1 over a set of transforms.  ``per_angle`` is a list of (mi_map, n_map).

    I starts at 0 and T-hat at the identity (no transform chosen, angle index -1);
    a transform replaces the best only when its I_T is strictly greater.  Also
    returns the top_k per-transform bests, by MI descending, earlier transform
    first among equals.
    """
    best = (-1, -1, 0.0, 0)   # (angle index, flat shift index, I, N)
    recs = []
    for t, (mi, n) in enumerate(per_angle):
        idx, i_t, n_t = gamma_argmax(mi, n, gamma)
        recs.append((t, idx, i_t, n_t))
        if i_t > best[2]:
            best = (t, idx, i_t, n_t)
    order = sorted(range(len(recs)), key=lambda k: (-recs[k][2], recs[k][0]))
    return best, [recs[k] for k in order[:top_k]]


def alg1_padded(A, M_A, B, M_B, K_A, K_B, gamma):
    """One transform of Alg. 1 with the ZERO-PAD step of Alg. 1.

    Pads A and M_A by p_i = ceil(|X_B|_i (1 - gamma)) zeros on both sides of
    each axis, computes the direct CMIF of (padded A, B), restricts it to X_S =
    the shifts at which B's whole domain lies inside padded A's, and takes the
    gamma-gated argmax there (max N over X_S; ties: lowest row-major index).
    Returns dict(dy, dx, mi, n, window=(dy_lo, dy_hi, dx_lo, dx_hi)) with the
    displacement relative to the UNPADDED A (the padding shifts chi by p).
    """
    A = np.asarray(A)
    H_A, W_A = A.shape
    H_B, W_B = np.asarray(B).shape
    py = int(np.ceil(H_B * (1.0 - gamma)))
    px = int(np.ceil(W_B * (1.0 - gamma)))
    Ap = np.zeros((H_A + 2 * py, W_A + 2 * px), dtype=A.dtype)
    Ap[py:py + H_A, px:px + W_A] = A
    Mp = np.zeros(Ap.shape, dtype=np.uint8)
    Mp[py:py + H_A, px:px + W_A] = 1 if M_A is None else np.asarray(M_A, dtype=np.uint8)
    ref = cmif(Ap, Mp, B, M_B, K_A, K_B)
    Hp, Wp = Ap.shape
    # padded-map row index = chi'_y + Hp - 1; B inside padded A: chi'_y in [H_B - Hp, 0]
    rows = np.arange(H_B - Hp, 1) + Hp - 1
    cols = np.arange(W_B - Wp, 1) + Wp - 1
    if rows.size == 0 or cols.size == 0:
        return None
    sub_mi = ref["mi"][np.ix_(rows, cols)]
    sub_n = ref["n"][np.ix_(rows, cols)]
    idx, mi, n = gamma_argmax(sub_mi, sub_n, gamma)
    i, j = divmod(idx, cols.size)
    # chi' = padded-map index - (Hp - 1); chi (unpadded A) = chi' + p
    dy = int(rows[i]) - (Hp - 1) + py
    dx = int(cols[j]) - (Wp - 1) + px
    win = (H_B - Hp + py, py, W_B - Wp + px, px)
    return dict(dy=dy, dx=dx, mi=mi, n=n, window=win, sub_mi=sub_mi, sub_n=sub_n)


def align_two_stage(A, M_A, B, M_B, K_A, K_B, n_grid, refine_u, gamma, padded=False, warp=None):
    """Two-stage rigid alignment (Sec. 3.6): Alg. 1 over theta_t = 2 pi t / n_grid,
    then over theta* + (2 u_i - 1) 2 pi / n_grid (theta* = the grid choice, 0 for
    the identity), keeping I and T-hat across the stages (strict >).

    Returns ((angle_idx, dy, dx, n, mi), theta); angle_idx = t for grid angles,
    n_grid + i for refinement angle i, -1 for the identity.  ``warp(B, M_B,
    theta) -> (B_theta, M_theta)`` replaces ``warp_nn`` when given (a test can
    pass the warped images of another implementation, so that count parity does
    not depend on rounding ties of the warp).
    """
    warp = warp or warp_nn

    def per_angle(theta):
        wB, wM = warp(B, M_B, theta)
        if padded:
            r = alg1_padded(A, M_A, wB, wM, K_A, K_B, gamma)
            return r["dy"], r["dx"], r["n"], r["mi"]
        ref = cmif(A, M_A, wB, wM, K_A, K_B)
        idx, mi, n = gamma_argmax(ref["mi"], ref["n"], gamma)
        C = ref["mi"].shape[1]
        i, j = divmod(idx, C)
        return i - (np.asarray(A).shape[0] - 1), j - (np.asarray(A).shape[1] - 1), n, mi

    best, theta_best = (-1, 0, 0, 0, 0.0), 0.0
    grid = [2.0 * np.pi * t / n_grid for t in range(n_grid)]
    for t, th in enumerate(grid):
        dy, dx, n, mi = per_angle(th)
        if mi > best[4]:
            best, theta_best = (t, dy, dx, n, mi), th
    base = theta_best
    for i, u in enumerate(refine_u):
        th = base + (2.0 * float(u) - 1.0) * 2.0 * np.pi / n_grid
        dy, dx, n, mi = per_angle(th)
        if mi > best[4]:
            best, theta_best = (n_grid + i, dy, dx, n, mi), th
    return best, theta_best


def nmi(A, M_A, B, M_B, K_A, K_B):
    """NMI map (H_A + H_B) / H_AB over the full shift range, from the direct
    method's per-shift entropies; 0 where N = 0 or H_AB = 0 (0/0 = 0)."""
    ref = cmif(A, M_A, B, M_B, K_A, K_B, entropies=True)
    ha, hb, hab = ref["ent"]
    out = np.zeros_like(hab)
    ok = hab > 0
    out[ok] = (ha[ok] + hb[ok]) / hab[ok]
    return dict(nmi=out, n=ref["n"], h_ab=hab)


def swmi(A, W_A, B, W_B, K_A, K_B):
    """Spatially weighted MI over the full shift range (Sec. 3.3), by the direct
    weighted histogram: at each chi every pixel pair (x, x + chi) with both weights
    > 0 adds W_A(x) W_B(x + chi) to bin (A(x), B(x + chi)); p = bins / N with N the
    total; MI = sum p log2(p / (p_a p_b)) (Eq. mi), 0 where N = 0.  W_* = None means
    all ones.  Returns dict(mi, nw) of shape (H_A + H_B - 1, W_A + W_B - 1)."""
    A = np.asarray(A, np.int64)
    B = np.asarray(B, np.int64)
    HA, WA = A.shape
    HB, WB = B.shape
    wa = np.ones(A.shape) if W_A is None else np.asarray(W_A, np.float64)
    wb = np.ones(B.shape) if W_B is None else np.asarray(W_B, np.float64)
    R, C = HA + HB - 1, WA + WB - 1
    mi = np.zeros((R, C))
    nw = np.zeros((R, C))
    for r in range(R):
        dy = r - (HA - 1)
        ya0, ya1 = max(0, -dy), min(HA, HB - dy)
        for c in range(C):
            dx = c - (WA - 1)
            xa0, xa1 = max(0, -dx), min(WA, WB - dx)
            if ya1 <= ya0 or xa1 <= xa0:
                continue
            a = A[ya0:ya1, xa0:xa1]
            b = B[ya0 + dy:ya1 + dy, xa0 + dx:xa1 + dx]
            w = wa[ya0:ya1, xa0:xa1] * wb[ya0 + dy:ya1 + dy, xa0 + dx:xa1 + dx]
            keep = (wa[ya0:ya1, xa0:xa1] > 0) & (wb[ya0 + dy:ya1 + dy, xa0 + dx:xa1 + dx] > 0)
            if not keep.any():
                continue
            if (a[keep] < 0).any() or (a[keep] >= K_A).any() or (b[keep] < 0).any() or (b[keep] >= K_B).any():
                raise OracleError("label outside [0, K) under a positive weight")
            joint = np.bincount(a[keep] * K_B + b[keep], weights=w[keep], minlength=K_A * K_B).reshape(K_A, K_B)
            n = joint.sum()
            nw[r, c] = n
            if n <= 0:
                continue
            p = joint / n
            pa = p.sum(axis=1, keepdims=True)
            pb = p.sum(axis=0, keepdims=True)
            nz = p > 0
            mi[r, c] = float((p[nz] * np.log2(p[nz] / (pa @ pb)[nz])).sum())
    return dict(mi=mi, nw=nw)


def cmif3(A, M_A, B, M_B, K_A, K_B):
    """CMIF of label volumes A (D_A x H_A x W_A) and B over every displacement
    chi = (dz, dy, dx) of the full linear range, by the direct method: the joint
    histogram of the voxel pairs (A(x), B(x + chi)) where both masks are 1, MI =
    sum p log2(p / (p_a p_b)) (Eq. mi), 0 where N = 0; and NMI = (H_A + H_B) / H_AB
    from the same histogram's entropies (Sec. 2.1), 0 where N = 0 or H_AB = 0.
    Returns dict(mi, n, nmi, h_ab) as maps of (D_A + D_B - 1) * (H_A + H_B - 1) rows
    (depth-offset major) by W_A + W_B - 1."""
    A = np.asarray(A, np.int64)
    B = np.asarray(B, np.int64)
    DA, HA, WA = A.shape
    DB, HB, WB = B.shape
    ma = np.ones(A.shape, bool) if M_A is None else np.asarray(M_A) != 0
    mb = np.ones(B.shape, bool) if M_B is None else np.asarray(M_B) != 0
    R2, C = HA + HB - 1, WA + WB - 1
    Dz = DA + DB - 1
    mi = np.zeros((Dz * R2, C))
    nmi_map = np.zeros((Dz * R2, C))
    hab_map = np.zeros((Dz * R2, C))
    n = np.zeros((Dz * R2, C), np.int64)

    def entropy(q):
        q = q[q > 0]
        return float(-(q * np.log2(q)).sum())

    def span(d, la, lb):
        return max(0, -d), min(la, lb - d)
    for zi in range(Dz):
        dz = zi - (DA - 1)
        z0, z1 = span(dz, DA, DB)
        for r in range(R2):
            dy = r - (HA - 1)
            y0, y1 = span(dy, HA, HB)
            for c in range(C):
                dx = c - (WA - 1)
                x0, x1 = span(dx, WA, WB)
                if z1 <= z0 or y1 <= y0 or x1 <= x0:
                    continue
                a = A[z0:z1, y0:y1, x0:x1]
                b = B[z0 + dz:z1 + dz, y0 + dy:y1 + dy, x0 + dx:x1 + dx]
                keep = ma[z0:z1, y0:y1, x0:x1] & mb[z0 + dz:z1 + dz, y0 + dy:y1 + dy, x0 + dx:x1 + dx]
                if not keep.any():
                    continue
                joint = np.bincount(a[keep] * K_B + b[keep], minlength=K_A * K_B).reshape(K_A, K_B)
                tot = int(joint.sum())
                n[zi * R2 + r, c] = tot
                p = joint / tot
                pa = p.sum(axis=1, keepdims=True)
                pb = p.sum(axis=0, keepdims=True)
                nz = p > 0
                mi[zi * R2 + r, c] = float((p[nz] * np.log2(p[nz] / (pa @ pb)[nz])).sum())
                h_ab = entropy(p.ravel())
                hab_map[zi * R2 + r, c] = h_ab
                if h_ab > 0:
                    nmi_map[zi * R2 + r, c] = (entropy(pa.ravel()) + entropy(pb.ravel())) / h_ab
    return dict(mi=mi, n=n, nmi=nmi_map, h_ab=hab_map)
