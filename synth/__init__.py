"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module draws random numbers and shapes them into density fields and test
vectors. It holds none of the method's arithmetic (no stiffness, no operator, no
solver, no policy): both sides receive the same arrays from here and compute
independently.

Element order everywhere is e = ex + nx*(ey + ny*ez) (x fastest), so a C-order
array of shape (nz, ny, nx) flattens to element order.

Recipes (stated for the workloads the paper's states are shaped like):

* ``uniform_density``   -- i.i.d. U[0,1) per element from NumPy ``default_rng(seed)``,
  the generator the paper names for its random states (Sec. 3.1, "Benchmark
  geometries").
* ``bernoulli_density`` -- the paper's hard-field stress state: u ~ U(0,1)^{n_e} from
  ``default_rng(seed)``; solid (1.0) iff u_e < q, else void (0.0) (Sec. 3.1).
* ``smoothed_gaussian_density`` -- white N(0,1) noise from ``default_rng(seed)``,
  Gaussian-smoothed with sigma cells (reflect boundary), then the ``floor_frac``
  lowest voxels (ties by element index) set to 0 and the rest to 1.
* ``optimised_like_density`` -- a smooth load-path-shaped field built from a few
  seeded, randomly placed tapered bars between the clamped face and the load
  point, blurred and thresholded to a target volume; then a seeded random
  ``floor_frac`` of voxels is forced to 0. A cheap stand-in for SIMP-optimised
  fields, which the paper does not publish (used where no SIMP-OC run is at hand).
* ``force_to_floor`` -- a seeded uniform-random choice of exactly
  floor(frac * n_e) voxels of a given field set to 0 ("forced to floor"); applied
  to a SIMP-OC design it gives the optimised-like states of the large and batched
  workloads (the SIMP-OC run itself is the method's arithmetic and happens in the
  library or in the oracle, never here).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "n_elements",
    "uniform_density",
    "bernoulli_density",
    "smoothed_gaussian_density",
    "optimised_like_density",
    "force_to_floor",
    "random_vector",
    "batch_grid_sizes",
]


def n_elements(nx: int, ny: int, nz: int) -> int:
    return int(nx) * int(ny) * int(nz)


def uniform_density(nx: int, ny: int, nz: int, seed: int) -> np.ndarray:
    """rho_hat_e ~ U[0,1) i.i.d., element order, float64."""
    rng = np.random.default_rng(seed)
    return rng.random(n_elements(nx, ny, nz))


def bernoulli_density(nx: int, ny: int, nz: int, seed: int, q: float) -> np.ndarray:
    """Solid (1) where u_e < q, void (0) elsewhere; u ~ U(0,1) from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    u = rng.random(n_elements(nx, ny, nz))
    return np.where(u < q, 1.0, 0.0)


def _threshold_lowest(field: np.ndarray, floor_frac: float) -> np.ndarray:
    """Binary field: the floor(floor_frac*n) lowest values -> 0, the rest -> 1.

    Ties are broken by element index (stable sort), so the result is unique.
    """
    flat = field.ravel()
    n = flat.size
    n_floor = int(np.floor(floor_frac * n))
    order = np.argsort(flat, kind="stable")
    out = np.ones(n, dtype=np.float64)
    out[order[:n_floor]] = 0.0
    return out


def smoothed_gaussian_density(nx: int, ny: int, nz: int, seed: int,
                              sigma: float = 2.0, floor_frac: float = 0.4) -> np.ndarray:
    """Smoothed-Gaussian random binary density with ``floor_frac`` of voxels at 0."""
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((nz, ny, nx))
    smooth = gaussian_filter(noise, sigma=sigma, mode="reflect")
    return _threshold_lowest(smooth, floor_frac)


def optimised_like_density(nx: int, ny: int, nz: int, seed: int,
                           volume: float = 0.3, floor_frac: float = 0.3,
                           n_bars: int = 10) -> np.ndarray:
    """Load-path-shaped smooth field, thresholded to ``volume``, with ``floor_frac`` forced to 0.

    Bars run from random points on the clamped x=0 face to points near the
    loaded tip (x = nx, y = ny/2, z = nz/2); each bar is a tube whose radius
    tapers from the support to the tip. The union is Gaussian-blurred (1 cell)
    and the top ``volume`` fraction of voxels kept solid (1), the rest 0. Then a
    seeded uniform-random ``floor_frac`` of all voxels is set to 0.
    """
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(seed)
    zc, yc, xc = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5,
                             np.arange(nx) + 0.5, indexing="ij")
    field = np.zeros((nz, ny, nx))
    tip = np.array([nx, ny / 2.0, nz / 2.0])
    for _ in range(n_bars):
        a = np.array([0.0, rng.uniform(0, ny), rng.uniform(0, nz)])
        b = tip + np.array([-rng.uniform(0, 0.25 * nx), rng.uniform(-0.2, 0.2) * ny,
                            rng.uniform(-0.2, 0.2) * nz])
        d = b - a
        L2 = float(d @ d)
        px, py, pz = xc - a[0], yc - a[1], zc - a[2]
        t = np.clip((px * d[0] + py * d[1] + pz * d[2]) / L2, 0.0, 1.0)
        qx, qy, qz = px - t * d[0], py - t * d[1], pz - t * d[2]
        dist = np.sqrt(qx * qx + qy * qy + qz * qz)
        r = (0.06 + 0.06 * (1.0 - t)) * ny
        field = np.maximum(field, np.clip(1.0 - dist / np.maximum(r, 1.0), 0.0, 1.0))
    field = gaussian_filter(field, sigma=1.0, mode="nearest")
    rho = _threshold_lowest(field, 1.0 - volume)  # lowest (1-volume) -> 0, rest -> 1
    kill = rng.random(rho.size) < floor_frac
    rho[kill] = 0.0
    return rho


def force_to_floor(rho: np.ndarray, frac: float, seed: int) -> np.ndarray:
    """A copy of rho with a seeded uniform-random set of exactly floor(frac * n) voxels
    set to 0 (the choice is the first floor(frac * n) entries of a permutation drawn
    from ``default_rng(seed)``)."""
    out = np.array(rho, dtype=np.float64, copy=True).ravel()
    rng = np.random.default_rng(seed)
    k = int(np.floor(frac * out.size))
    out[rng.permutation(out.size)[:k]] = 0.0
    return out


def random_vector(n: int, seed: int) -> np.ndarray:
    """U(-1,1) float64 test vector."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, n)


def batch_grid_sizes(n_states: int = 102):
    """Uneven grid sizes for a batch of frozen states: nx in {32,48,64,80},
    ny = nz = nx/2, assigned round-robin (every size divisible by 8)."""
    sizes = (32, 48, 64, 80)
    return [(sizes[i % 4], sizes[i % 4] // 2, sizes[i % 4] // 2) for i in range(n_states)]


def mlp_init(seed: int, sizes=(6, 32, 32, 4)) -> np.ndarray:
    """Initial weights for the selector MLP (flat, float32): W ~ N(0, 1/fan_in), b = 0,
    in the layout W1, b1, W2, b2, W3, b3 ([out][in] rows)."""
    rng = np.random.default_rng(seed)
    parts = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        parts.append(rng.normal(0.0, 1.0 / np.sqrt(a), size=(b, a)).ravel())
        parts.append(np.zeros(b))
    return np.concatenate(parts).astype(np.float32)


def epoch_permutations(n: int, epochs: int, seed: int) -> np.ndarray:
    """epochs concatenated random permutations of range(n) (minibatch order)."""
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.permutation(n) for _ in range(epochs)]).astype(np.int32)


def selector_training_states(n: int, dims, seed: int, designs=None):
    """A mix of states for selector training, in turn: Bernoulli hard fields with solid
    probability q ~ U(0.15, 0.6); smoothed-Gaussian fields with floor fraction
    ~ U(0.1, 0.6) and sigma in {1, 2, 3}; optimised-like fields with forced-floor
    fraction ~ U(0.1, 0.5): with ``designs`` (a list of SIMP-OC designs of this size)
    a seeded choice among them passed through ``force_to_floor``, else
    ``optimised_like_density`` with volume ~ U(0.2, 0.4)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    out = []
    for i in range(n):
        s = int(rng.integers(0, 2**31 - 1))
        if i % 3 == 0:
            out.append(bernoulli_density(nx, ny, nz, s, float(rng.uniform(0.15, 0.6))))
        elif i % 3 == 1:
            out.append(smoothed_gaussian_density(nx, ny, nz, s, float(rng.choice([1.0, 2.0, 3.0])),
                                                 float(rng.uniform(0.1, 0.6))))
        elif designs:
            base = designs[int(rng.integers(0, len(designs)))]
            out.append(force_to_floor(base, float(rng.uniform(0.1, 0.5)), s))
        else:
            out.append(optimised_like_density(nx, ny, nz, s, float(rng.uniform(0.2, 0.4)),
                                              float(rng.uniform(0.1, 0.5))))
    return out
