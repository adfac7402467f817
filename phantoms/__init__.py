"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module draws geometry and random numbers only.  It holds none of the
Lippmann-Schwinger arithmetic: it returns refractive-index *contrasts* ``dn``
(so that eta = eta_b + dn), illumination *directions* (unit vectors) and
complex Gaussian noise.  The conversion of ``dn`` to a scattering potential,
of a direction to a wave vector and everything after that is done separately
by the oracle and by the CUDA library.

Volumes are numpy arrays indexed ``[z, y, x]`` (x fastest).  Voxel ``(i, j, k)``
(x, y, z array indices) sits at ``h * (i - nx/2 + 1, j - ny/2 + 1, k - nz/2 + 1)``,
the centred index set of the paper's DFT (Sec. 1.4 and Theorem 1).

The paper's own data (DDA-simulated red blood cells, a measured yeast cell)
is not available; these generators stand in for it with the shapes and
contrasts of the paper's workloads (Sec. 5 and Fig. 3).
"""
from __future__ import annotations

import numpy as np

SEED_PHANTOM = 13844
SEED_NOISE = 13845

# Physical set-up shared by every workload: vacuum wavelength (um), background
# index (water-like medium) and voxel size lambda/8.
LAMBDA_UM = 0.532
ETA_B = 1.333
VOXEL_UM = LAMBDA_UM / 8.0


def centred_coords(n: int) -> np.ndarray:
    """Integer centred indices ``i - n/2 + 1`` for array indices ``i = 0..n-1``."""
    return np.arange(n, dtype=np.float64) - (n // 2) + 1.0


def voxel_centres(shape):
    """Centred integer coordinates (z, y, x) broadcastable over ``shape=(nz, ny, nx)``."""
    nz, ny, nx = shape
    z = centred_coords(nz)[:, None, None]
    y = centred_coords(ny)[None, :, None]
    x = centred_coords(nx)[None, None, :]
    return z, y, x


def sphere(shape, radius_vox: float, dn: float, centre=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Homogeneous sphere sampled at voxel centres (binary inside test).

    ``centre`` is given in centred voxel units (z, y, x); (0, 0, 0) is the
    grid's origin voxel.
    """
    z, y, x = voxel_centres(shape)
    cz, cy, cx = centre
    r2 = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2
    return np.where(r2 <= radius_vox * radius_vox, dn, 0.0).astype(np.float64)


def sphere_fraction(shape, radius_vox: float, dn: float, centre=(0.0, 0.0, 0.0), sub: int = 4) -> np.ndarray:
    """Sphere with ``dn`` weighted by the voxel's volume fraction (``sub**3`` sub-samples)."""
    z, y, x = voxel_centres(shape)
    cz, cy, cx = centre
    acc = np.zeros(shape, dtype=np.float64)
    offs = (np.arange(sub) + 0.5) / sub - 0.5
    for oz in offs:
        for oy in offs:
            for ox in offs:
                r2 = (x + ox - cx) ** 2 + (y + oy - cy) ** 2 + (z + oz - cz) ** 2
                acc += (r2 <= radius_vox * radius_vox)
    return dn * acc / float(sub ** 3)


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniformly distributed rotation matrix (QR of a Gaussian matrix, sign-fixed)."""
    a = rng.standard_normal((3, 3))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _ellipsoid_mask(shape, centre, semi_axes, rot):
    z, y, x = voxel_centres(shape)
    cz, cy, cx = centre
    d = np.stack(np.broadcast_arrays(x - cx, y - cy, z - cz), axis=-1)  # (..., 3) in x,y,z
    local = d @ rot  # coordinates along the ellipsoid's principal axes
    a, b, c = semi_axes
    q = (local[..., 0] / a) ** 2 + (local[..., 1] / b) ** 2 + (local[..., 2] / c) ** 2
    return q <= 1.0


def random_ellipsoids(shape, count: int = 20, rmin: float = 4.0, rmax: float = 20.0,
                      dn_max: float = 0.05, margin: int = 2, seed: int = SEED_PHANTOM) -> np.ndarray:
    """``count`` randomly rotated ellipsoids, contrast uniform in [0, dn_max], max on overlap.

    Semi-axes are uniform in [rmin, rmax] voxels; each centre is uniform over the
    positions that keep the ellipsoid's bounding sphere ``margin`` voxels inside
    the grid.
    """
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    out = np.zeros(shape, dtype=np.float64)
    for _ in range(count):
        semi = rng.uniform(rmin, rmax, size=3)
        rot = _random_rotation(rng)
        dn = rng.uniform(0.0, dn_max)
        rb = float(semi.max()) + margin
        centre = []
        for n in (nz, ny, nx):
            lo = -(n // 2) + 1 + rb
            hi = (n // 2) - rb
            if hi < lo:
                lo = hi = 0.5 * (-(n // 2) + 1 + (n // 2))
            centre.append(rng.uniform(lo, hi))
        mask = _ellipsoid_mask(shape, tuple(centre), tuple(semi), rot)
        out = np.where(mask, np.maximum(out, dn), out)
    return out


def cell(shape, seed: int = SEED_PHANTOM, shell=(52.0, 44.0, 36.0), nucleus=(18.0, 16.0, 14.0),
         nucleus_offset_x: float = 8.0, n_granules: int = 50, dn_shell: float = 0.03,
         dn_nucleus: float = 0.05, dn_granule: float = 0.08, scale: float = 1.0) -> np.ndarray:
    """Cell-like phantom: cytoplasm ellipsoid, offset nucleus and small dense granules.

    Sizes are in voxels for a 128 x 128 x 96 grid and multiplied by ``scale``
    for other grids.  Granules (radius uniform in [2, 4] voxels) are placed at
    random inside the cytoplasm and outside the nucleus.  Max on overlap.
    """
    rng = np.random.default_rng(seed)
    eye = np.eye(3)
    sa = tuple(s * scale for s in shell)
    na = tuple(s * scale for s in nucleus)
    ncen = (0.0, 0.0, nucleus_offset_x * scale)
    out = np.where(_ellipsoid_mask(shape, (0.0, 0.0, 0.0), sa, eye), dn_shell, 0.0)
    inside_nucleus = _ellipsoid_mask(shape, ncen, na, eye)
    out = np.where(inside_nucleus, np.maximum(out, dn_nucleus), out)
    z, y, x = voxel_centres(shape)
    placed = 0
    tries = 0
    while placed < n_granules and tries < 100000:
        tries += 1
        r = rng.uniform(2.0, 4.0) * scale
        c = np.array([rng.uniform(-s, s) for s in (sa[2], sa[1], sa[0])])  # z, y, x
        # centre must be inside the shell (with the granule fully inside) and outside the nucleus
        qs = (c[2] / (sa[0] - r)) ** 2 + (c[1] / (sa[1] - r)) ** 2 + (c[0] / (sa[2] - r)) ** 2 if min(sa) > r else 2.0
        qn = ((c[2] - ncen[2]) / (na[0] + r)) ** 2 + ((c[1] - ncen[1]) / (na[1] + r)) ** 2 + ((c[0] - ncen[0]) / (na[2] + r)) ** 2
        if qs > 1.0 or qn <= 1.0:
            continue
        mask = (x - c[2]) ** 2 + (y - c[1]) ** 2 + (z - c[0]) ** 2 <= r * r
        out = np.where(mask, np.maximum(out, dn_granule), out)
        placed += 1
    return out.astype(np.float64)


def cone_directions(count: int, na: float = 0.8, eta_b: float = ETA_B) -> np.ndarray:
    """Unit propagation directions on a cone of numerical aperture ``na`` about +z.

    ``sin(theta) = na / eta_b``, azimuths ``phi_q = 2 pi q / count`` (Fig. 1).
    Returns ``(count, 3)`` in (x, y, z) order.  ``count == 1`` with ``na == 0``
    gives the on-axis wave.
    """
    s = na / eta_b
    c = np.sqrt(max(0.0, 1.0 - s * s))
    phi = 2.0 * np.pi * np.arange(count) / max(count, 1)
    return np.stack([s * np.cos(phi), s * np.sin(phi), np.full(count, c)], axis=1)


def complex_normal(shape, seed: int = SEED_NOISE) -> np.ndarray:
    """i.i.d. complex Gaussian samples ``xi_1 + i xi_2`` with unit-variance parts."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def random_field(shape, seed: int) -> np.ndarray:
    """Generic complex test vector (complex Gaussian)."""
    return complex_normal(shape, seed)


def random_potential_like(shape, seed: int, dn_max: float = 0.05) -> np.ndarray:
    """Smooth-ish random contrast in [0, dn_max] (for operator tests, not physics)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, dn_max, size=shape)
