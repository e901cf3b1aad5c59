"""Seeded synthetic label images shaped like the paper's workloads.

This module only *makes inputs*.  It holds none of the CMIF arithmetic
(no histograms, no entropies, no transforms, no image warping); both the
CPU oracle and the CUDA library consume what it returns, and neither
shares code with the other.

The paper's datasets (aerial, cytological and histological image pairs,
Sec. 5) are not available here, so piecewise-constant Voronoi label maps
stand in for quantised images: the paper quantises each image into k
labels with k-means (Sec. 3.6), which yields exactly such label maps with
k in {8, 16, 32} (Sec. 5.1).  Masks follow the paper's ROI masks
(Sec. 3.1) and the circular masks of its evaluation (Sec. 5.2).

Every generator takes a ``numpy.random.Generator``; a whole workload is
reproducible from one integer seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.spatial import cKDTree

__all__ = [
    "LabelField", "make_field", "permutation", "label_noise", "disc_mask",
    "hole_mask", "ones_mask", "planted_pair", "make_workload", "WORKLOADS",
]


@dataclass
class LabelField:
    """A continuous piecewise-constant label field on the plane.

    ``label_at(rows, cols)`` returns the label of the nearest seed (Euclidean)
    at arbitrary real coordinates.  Sampling the field on the integer grid
    gives a Voronoi label image; sampling it on a rotated/shifted grid gives
    the same scene seen under a rigid transform, without resampling an image.
    """
    seeds: np.ndarray          # (n, 2) float64, (row, col)
    labels: np.ndarray         # (n,) int32 label of each cell
    tree: cKDTree = field(repr=False, default=None)

    def __post_init__(self):
        if self.tree is None:
            self.tree = cKDTree(self.seeds)

    def label_at(self, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
        pts = np.stack([np.asarray(rows, np.float64).ravel(),
                        np.asarray(cols, np.float64).ravel()], axis=1)
        _, idx = self.tree.query(pts, k=1)
        return self.labels[idx].reshape(np.shape(rows)).astype(np.int32)

    def relabel(self, rng: np.random.Generator, K: int) -> "LabelField":
        """Same cells, fresh uniform labels in [0, K) (a second modality)."""
        return LabelField(self.seeds, rng.integers(0, K, len(self.labels)).astype(np.int32), self.tree)

    def image(self, H: int, W: int, jitter: np.ndarray | None = None) -> np.ndarray:
        r, c = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
        if jitter is not None:
            r = r + jitter[0]
            c = c + jitter[1]
        return self.label_at(r, c)


def make_field(rng: np.random.Generator, H: int, W: int, n_cells: int, K: int) -> LabelField:
    """Voronoi field: seeds uniform over the H x W image, cell labels uniform in [0, K)."""
    seeds = np.stack([rng.uniform(0, H, n_cells), rng.uniform(0, W, n_cells)], axis=1)
    labels = rng.integers(0, K, n_cells).astype(np.int32)
    return LabelField(seeds, labels)


def permutation(rng: np.random.Generator, K: int) -> np.ndarray:
    return rng.permutation(K).astype(np.int32)


def label_noise(rng: np.random.Generator, img: np.ndarray, p: float, K: int) -> np.ndarray:
    """Each pixel independently, with probability p, gets a label uniform in [0, K)."""
    out = img.copy()
    hit = rng.random(img.shape) < p
    out[hit] = rng.integers(0, K, int(hit.sum()))
    return out


def ones_mask(H: int, W: int) -> np.ndarray:
    return np.ones((H, W), np.uint8)


def disc_mask(H: int, W: int, r: float) -> np.ndarray:
    """1 inside the centred disc (y - cy)^2 + (x - cx)^2 <= r^2, cy = (H-1)/2, cx = (W-1)/2."""
    y, x = np.meshgrid(np.arange(H) - (H - 1) / 2.0, np.arange(W) - (W - 1) / 2.0, indexing="ij")
    return ((y * y + x * x) <= r * r).astype(np.uint8)


def hole_mask(rng: np.random.Generator, H: int, W: int, n_holes: int = 5,
              area=(0.02, 0.05), aspect=(0.5, 2.0)) -> np.ndarray:
    """All-ones mask with axis-aligned rectangular holes (value 0)."""
    m = np.ones((H, W), np.uint8)
    for _ in range(n_holes):
        a = rng.uniform(*area) * H * W
        asp = rng.uniform(*aspect)
        h = max(1, min(H, int(round(math.sqrt(a * asp)))))
        w = max(1, min(W, int(round(a / h))))
        y0 = int(rng.integers(0, H - h + 1))
        x0 = int(rng.integers(0, W - w + 1))
        m[y0:y0 + h, x0:x0 + w] = 0
    return m


def planted_pair(rng, H, W, n_cells, K_A, K_B, shift, noise, angle_deg=0.0,
                 jitter=False, same_labels=False):
    """Reference A and floating B of one scene, B seen under a planted transform.

    A(x) = f_A(x) for the field f_A.  B is sampled so that rotating B by
    ``angle_deg`` about its centre and then shifting by chi* = ``shift``
    (row, col) lands it on A: B(s) = g(R(s - c) + c - chi*), where g is the
    same cells relabelled (K_B labels, or a permutation of A's labels when
    ``same_labels``) and R the rotation by angle_deg, counter-clockwise on
    screen with rows pointing down.  With angle 0 this is B(y) = g(y - chi*),
    whose CMIF peaks at chi = chi*.
    """
    fA = make_field(rng, H, W, n_cells, K_A)
    if same_labels:
        assert K_A == K_B
        perm = permutation(rng, K_B)
        fB = LabelField(fA.seeds, perm[fA.labels], fA.tree)
    else:
        fB = fA.relabel(rng, K_B)
    A = fA.image(H, W)
    th = math.radians(angle_deg)
    cr, cc = (H - 1) / 2.0, (W - 1) / 2.0
    r, c = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    u, v = c - cc, r - cr
    pc = cc + u * math.cos(th) + v * math.sin(th) - shift[1]
    pr = cr - u * math.sin(th) + v * math.cos(th) - shift[0]
    if jitter:
        pr = pr + rng.uniform(-0.5, 0.5, pr.shape)
        pc = pc + rng.uniform(-0.5, 0.5, pc.shape)
    B = fB.label_at(pr, pc)
    if noise > 0:
        B = label_noise(rng, B, noise, K_B)
    return A.astype(np.int32), B.astype(np.int32)


# The five workloads, by name, with the offset added to the seed for each (so
# that every workload draws its own stream).
WORKLOADS = {
    "plain-64x64-K8": 1000,
    "single-256x256-K16": 2000,
    "single-1024x1024-K16": 3000,
    "rotation-512x512-K16-64angles": 4000,
    "uneven-batch-128pairs": 5000,
}


def make_workload(name: str, seed: int = 2106_14699, scale: float = 1.0) -> dict:
    """Inputs for one of the WORKLOADS.  ``scale`` < 1 shrinks sides (test-sized variants).

    Returns a dict with A, M_A, B, M_B (numpy), K_A, K_B and the planted truth.
    "uneven-batch-128pairs" returns {"pairs": [...]} with one dict per pair.
    """
    if name not in WORKLOADS:
        raise ValueError(f"unknown workload {name!r}")
    rng = np.random.default_rng(seed + WORKLOADS[name])
    s = lambda n: max(8, int(round(n * scale)))
    if name == "plain-64x64-K8":
        H = W = s(64)
        lim = max(1, int(round(12 * min(1.0, scale))))
        d = tuple(int(v) for v in rng.integers(-lim, lim + 1, 2))
        K = 8
        fA = make_field(rng, H, W, 40, K)
        A = fA.image(H, W)
        perm = permutation(rng, K)
        B = label_noise(rng, np.roll(perm[A], d, axis=(0, 1)).astype(np.int32), 0.05, K)
        return dict(A=A, M_A=ones_mask(H, W), B=B, M_B=disc_mask(H, W, 28 * H / 64.0),
                    K_A=K, K_B=K, shift=d, name=name)
    if name in ("single-256x256-K16", "single-1024x1024-K16"):
        small = name == "single-256x256-K16"
        H = W = s(256 if small else 1024)
        K = 16
        n_cells = 300 if small else 2000
        lim = max(1, int(round(40 * min(1.0, scale))))
        d = tuple(int(v) for v in rng.integers(-lim, lim + 1, 2))
        A, B = planted_pair(rng, H, W, n_cells, K, K, d, 0.10, jitter=not small, same_labels=True)
        if small:
            MA, MB = hole_mask(rng, H, W), hole_mask(rng, H, W)
        else:
            MA, MB = ones_mask(H, W), ones_mask(H, W)
        return dict(A=A, M_A=MA, B=B, M_B=MB, K_A=K, K_B=K, shift=d, name=name)
    if name == "rotation-512x512-K16-64angles":
        H = W = s(512)
        K = 16
        shift = (int(round(-23 * scale)), int(round(61 * scale)))
        A, B = planted_pair(rng, H, W, max(40, int(1200 * scale * scale)), K, K, shift, 0.0,
                            angle_deg=37.5, same_labels=True)
        n_angles = 64
        angles = np.arange(n_angles) * (2 * math.pi / n_angles)
        return dict(A=A, M_A=ones_mask(H, W), B=B, M_B=ones_mask(H, W), K_A=K, K_B=K,
                    shift=shift, angle_deg=37.5, angles=angles, name=name)
    # uneven-batch-128pairs
    pairs = []
    n_pairs = 128 if scale >= 1.0 else max(2, int(round(128 * scale)))
    lo, hi = math.log(s(96)), math.log(s(1536))
    for p in range(n_pairs):
        H = int(round(math.exp(rng.uniform(lo, hi))))
        W = int(round(math.exp(rng.uniform(lo, hi))))
        K_A = int(rng.choice([8, 16, 24]))
        K_B = int(rng.choice([8, 16, 24]))
        th = float(rng.uniform(0, 360))
        lim = max(1, min(H, W) // 8)
        d = tuple(int(v) for v in rng.integers(-lim, lim + 1, 2))
        n_cells = max(20, int(H * W / 500))
        A, B = planted_pair(rng, H, W, n_cells, K_A, K_B, d, 0.10, angle_deg=th)
        angles = np.concatenate([[math.radians(th)], rng.uniform(0, 2 * math.pi, 3)])
        pairs.append(dict(A=A, M_A=hole_mask(rng, H, W), B=B, M_B=hole_mask(rng, H, W),
                          K_A=K_A, K_B=K_B, shift=d, angle_deg=th, angles=angles))
    return dict(pairs=pairs, name=name)
