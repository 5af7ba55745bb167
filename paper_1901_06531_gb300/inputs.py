"""Seeded synthetic inputs shared by the CUDA path, the tests and the bench.

This module generates microstructures, orientations, scale fields, load
histories and random tensor fields.  It holds none of the homogenization
arithmetic (no transforms, no projector, no constitutive law): both the CUDA
library and the CPU oracle receive its arrays as plain inputs.

Conventions used everywhere in the project:

* voxel fields are ``numpy`` arrays indexed ``[z, y, x]`` (x fastest);
* tensor fields are ``[c, z, y, x]`` with ``c = 3*i + j`` for component ij;
* voxels are unit cubes, voxel centres sit at ``(x + 1/2, y + 1/2, z + 1/2)``;
* a load history is ``(mask, target)``, both ``(nsteps, 9)``: ``mask[k, c] = 1``
  means component c of the macroscopic first Piola stress is prescribed at step
  k (target holds P-bar), ``0`` means the macroscopic deformation gradient
  component is prescribed (target holds F-bar).  This is the per-component
  stress/strain control of Section 2.3 (mixed control).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "periodic_sphere_phase", "centred_sphere", "rsa_spheres", "voronoi",
    "random_rotations", "lognormal_scale", "random_F", "random_field",
    "history_uniaxial_stress_ramp", "history_mixed_strain11",
    "history_cyclic_stress", "laminate_phase", "fix_rotation", "random_control", "batch_of_cells",
    "particle_rve", "history_case1", "history_case2", "history_case3", "history_case4",
]


def _grid_centres(shape):
    nz, ny, nx = shape
    z = np.arange(nz) + 0.5
    y = np.arange(ny) + 0.5
    x = np.arange(nx) + 0.5
    return z, y, x


def _min_image(d, length):
    d = np.abs(d)
    return np.minimum(d, length - d)


def periodic_sphere_phase(shape, centres, radius):
    """Phase map: 1 inside any periodic sphere (min-image distance <= radius)."""
    nz, ny, nx = shape
    z, y, x = _grid_centres(shape)
    phase = np.zeros(shape, dtype=np.int32)
    for (cx, cy, cz) in centres:
        dz = _min_image(z - cz, nz)[:, None, None]
        dy = _min_image(y - cy, ny)[None, :, None]
        dx = _min_image(x - cx, nx)[None, None, :]
        phase[(dx * dx + dy * dy + dz * dz) <= radius * radius] = 1
    return phase


def centred_sphere(n, r_frac=0.25):
    """One sphere of radius r_frac*n centred in an n^3 cell (two-phase RVE)."""
    c = n / 2.0
    return periodic_sphere_phase((n, n, n), [(c, c, c)], r_frac * n)


def rsa_spheres(shape, radius, vf, seed):
    """Random sequential addition of non-overlapping periodic spheres.

    Centres are drawn uniformly in the cell; a candidate is accepted when its
    periodic centre distance to every accepted sphere is >= 2*radius.  Spheres
    are added until the voxel volume fraction of phase 1 reaches ``vf``.
    Returns (phase, centres).
    """
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    lengths = np.array([nx, ny, nz], dtype=np.float64)
    centres = []
    phase = np.zeros(shape, dtype=np.int32)
    z, y, x = _grid_centres(shape)
    target = vf * phase.size
    count = 0
    attempts = 0
    while count < target:
        attempts += 1
        if attempts > 200000:
            raise RuntimeError("rsa_spheres: could not reach the volume fraction")
        c = rng.random(3) * lengths
        if centres:
            d = np.abs(np.asarray(centres) - c)
            d = np.minimum(d, lengths - d)
            if np.min(np.sum(d * d, axis=1)) < (2.0 * radius) ** 2:
                continue
        centres.append(c)
        dz = _min_image(z - c[2], nz)[:, None, None]
        dy = _min_image(y - c[1], ny)[None, :, None]
        dx = _min_image(x - c[0], nx)[None, None, :]
        inside = (dx * dx + dy * dy + dz * dz) <= radius * radius
        count += int(np.count_nonzero(inside & (phase == 0)))
        phase[inside] = 1
    return phase, np.asarray(centres)


def voronoi(shape, ngrains, seed):
    """Periodic Voronoi tessellation: each voxel takes the index of the nearest
    of ``ngrains`` uniform seeds (min-image distance; ties go to the lower
    index).  Returns (grain_id int32 [z,y,x], seeds (ngrains, 3) as x,y,z)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    lengths = np.array([nx, ny, nz], dtype=np.float64)
    seeds = rng.random((ngrains, 3)) * lengths
    z, y, x = _grid_centres(shape)
    grain = np.empty(shape, dtype=np.int32)
    for iz in range(nz):
        best = np.full((ny, nx), np.inf)
        arg = np.zeros((ny, nx), dtype=np.int32)
        dz2 = _min_image(z[iz] - seeds[:, 2], nz) ** 2
        for g in range(ngrains):
            dy = _min_image(y - seeds[g, 1], ny)[:, None]
            dx = _min_image(x - seeds[g, 0], nx)[None, :]
            d2 = dx * dx + dy * dy + dz2[g]
            better = d2 < best
            best = np.where(better, d2, best)
            arg = np.where(better, g, arg)
        grain[iz] = arg
    return grain, seeds


def laminate_phase(shape, axis, n_a, offset=0):
    """Layered two-phase map: phase 1 in ``n_a`` consecutive voxel layers normal
    to ``axis`` (0=x, 1=y, 2=z) starting at ``offset``, phase 0 elsewhere."""
    nz, ny, nx = shape
    n = (nx, ny, nz)[axis]
    layer = np.zeros(n, dtype=np.int32)
    idx = (np.arange(n_a) + offset) % n
    layer[idx] = 1
    if axis == 0:
        return np.broadcast_to(layer[None, None, :], shape).astype(np.int32)
    if axis == 1:
        return np.broadcast_to(layer[None, :, None], shape).astype(np.int32)
    return np.broadcast_to(layer[:, None, None], shape).astype(np.int32)


def random_rotations(count, seed):
    """Uniformly distributed rotation matrices (Shoemake's uniform unit
    quaternions, Graphics Gems III, 1992).  Returns (count, 3, 3)."""
    rng = np.random.default_rng(seed)
    u1, u2, u3 = rng.random((3, count))
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    w = a * np.sin(2 * np.pi * u2)
    xq = a * np.cos(2 * np.pi * u2)
    yq = b * np.sin(2 * np.pi * u3)
    zq = b * np.cos(2 * np.pi * u3)
    R = np.empty((count, 3, 3))
    R[:, 0, 0] = 1 - 2 * (yq * yq + zq * zq)
    R[:, 0, 1] = 2 * (xq * yq - zq * w)
    R[:, 0, 2] = 2 * (xq * zq + yq * w)
    R[:, 1, 0] = 2 * (xq * yq + zq * w)
    R[:, 1, 1] = 1 - 2 * (xq * xq + zq * zq)
    R[:, 1, 2] = 2 * (yq * zq - xq * w)
    R[:, 2, 0] = 2 * (xq * zq - yq * w)
    R[:, 2, 1] = 2 * (yq * zq + xq * w)
    R[:, 2, 2] = 1 - 2 * (xq * xq + yq * yq)
    return R


def lognormal_scale(shape, sigma, seed):
    """Per-voxel stiffness scale s = exp(sigma*z - sigma^2/2), z iid N(0,1)
    (unit mean)."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(shape)
    return np.exp(sigma * z - 0.5 * sigma * sigma)


def random_F(shape, seed, amp=0.05):
    """Deformation-gradient field F = I + amp*U(-1,1) per component, [9,z,y,x]."""
    rng = np.random.default_rng(seed)
    F = amp * (2.0 * rng.random((9,) + tuple(shape)) - 1.0)
    F[0] += 1.0
    F[4] += 1.0
    F[8] += 1.0
    return F


def random_field(shape, seed, amp=1.0):
    """Tensor field with iid U(-amp, amp) components, [9,z,y,x]."""
    rng = np.random.default_rng(seed)
    return amp * (2.0 * rng.random((9,) + tuple(shape)) - 1.0)


def history_uniaxial_stress_ramp(nsteps, p11_end):
    """All nine components stress controlled; P11 ramps linearly to p11_end,
    every other P-bar component is 0."""
    mask = np.ones((nsteps, 9), dtype=np.uint8)
    target = np.zeros((nsteps, 9))
    target[:, 0] = p11_end * np.arange(1, nsteps + 1) / nsteps
    return mask, target


def history_mixed_strain11(nsteps, f11_end):
    """Mixed control: F11 ramps linearly to f11_end (strain controlled), the
    other eight components are stress free (P-bar = 0)."""
    mask = np.ones((nsteps, 9), dtype=np.uint8)
    mask[:, 0] = 0
    target = np.zeros((nsteps, 9))
    target[:, 0] = 1.0 + (f11_end - 1.0) * np.arange(1, nsteps + 1) / nsteps
    return mask, target


def history_cyclic_stress(nsteps, amplitude):
    """All nine components stress controlled; P11 follows a triangle wave
    0 -> +a -> -a -> 0 over ``nsteps`` equal increments (nsteps divisible by
    4); every other P-bar component is 0."""
    if nsteps % 4:
        raise ValueError("nsteps must be a multiple of 4")
    q = nsteps // 4
    t = np.arange(1, nsteps + 1)
    inc = amplitude / q
    p = np.where(t <= q, t * inc,
                 np.where(t <= 3 * q, amplitude - (t - q) * inc,
                          -amplitude + (t - 3 * q) * inc))
    mask = np.ones((nsteps, 9), dtype=np.uint8)
    target = np.zeros((nsteps, 9))
    target[:, 0] = p
    return mask, target


def fix_rotation(mask, target):
    """Replace the prescribed stress on components 12, 13 and 23 by a
    prescribed zero deformation-gradient component.  With F-bar upper
    off-diagonals held at zero the rigid rotation of the cell is fixed; this
    is the control pattern of the paper's load case (1) in Sec. 3.1.  Returns
    new (mask, target) arrays."""
    mask = np.array(mask, dtype=np.uint8, copy=True)
    target = np.array(target, dtype=np.float64, copy=True)
    for c in (1, 2, 5):
        mask[:, c] = 0
        target[:, c] = 0.0
    return mask, target


def random_control(nsteps, rng, amp=0.02):
    """Random mixed control: each component stress controlled with probability
    1/2 (at least one strain-controlled component); a rotation plane whose two
    off-diagonal components would both be stress controlled gets its upper
    component (12, 13 or 23) strain controlled at zero, so that no rigid
    rotation is left free.  Strain-controlled components ramp linearly from
    the identity by amp * U(-1, 1) over the steps; every prescribed stress is
    zero.  Returns (mask, target), (nsteps, 9) each."""
    m = (rng.random(9) < 0.5).astype(np.uint8)
    if m.all():
        m[rng.integers(0, 9)] = 0
    u = rng.uniform(-1.0, 1.0, 9)
    eye = np.array([1.0, 0, 0, 0, 1.0, 0, 0, 0, 1.0])
    zero_strain = np.zeros(9, dtype=bool)
    for up, lo in ((1, 3), (2, 6), (5, 7)):
        if m[up] and m[lo]:
            m[up] = 0
            zero_strain[up] = True
    t = np.arange(1, nsteps + 1)[:, None] / nsteps
    target = np.where(m[None, :] == 1, 0.0, eye[None, :] + amp * u[None, :] * t)
    target[:, zero_strain] = 0.0
    return np.tile(m, (nsteps, 1)), target


def batch_of_cells(count, seed, sizes=(32, 48, 64, 96), nsteps=4):
    """The batched workload: `count` sphere-particle neo-Hookean cells with
    grid sizes drawn from `sizes`, particle volume fraction U(0.1, 0.3),
    stiffness contrast U(5, 50) (matrix mu = 1, lam = 2), sphere radius n/12,
    and random mixed control (random_control).  Returns a list of dicts."""
    rng = np.random.default_rng(seed)
    cells = []
    for i in range(count):
        n = int(rng.choice(sizes))
        vf = rng.uniform(0.1, 0.3)
        contrast = rng.uniform(5.0, 50.0)
        phase, _ = rsa_spheres((n, n, n), n / 12.0, vf, int(rng.integers(1 << 30)))
        params = np.array([[1.0, 2.0], [contrast, 2.0 * contrast]])
        mask, target = random_control(nsteps, rng)
        cells.append({"n": n, "phase": phase, "params": params, "mask": mask, "target": target,
                      "vf": vf, "contrast": contrast})
    return cells


# ----------------------------------------------------------------------------
# The load cases of the paper's Sec. 3 (control cases (1)-(4)) and its
# particle-reinforced cell.

def particle_rve(n, seed, count=4, vf=0.2):
    """Stand-in for the paper's particle-reinforced cell (Sec. 3.1): `count`
    non-overlapping periodic spheres of equal radius whose volumes add up to
    the fraction `vf` of an n^3 cell (radius n (3 vf / (4 pi count))^(1/3)),
    placed by random sequential addition.  Returns the phase map (1 inside
    the particles)."""
    r = n * (3.0 * vf / (4.0 * np.pi * count)) ** (1.0 / 3.0)
    rng = np.random.default_rng(seed)
    lengths = np.array([n, n, n], dtype=np.float64)
    centres = []
    attempts = 0
    while len(centres) < count:
        attempts += 1
        if attempts > 100000:
            raise RuntimeError("particle_rve: could not place the particles")
        c = rng.random(3) * lengths
        if centres:
            d = np.abs(np.asarray(centres) - c)
            d = np.minimum(d, lengths - d)
            if np.min(np.sum(d * d, axis=1)) < (2.0 * r) ** 2:
                continue
        centres.append(c)
    return periodic_sphere_phase((n, n, n), [tuple(c) for c in centres], r)


def history_case1(nsteps, lambda_end):
    """Case (1), a uniaxial stress test in mixed control: F11 ramps to
    1 + lambda_end (lambda_end read as an engineering strain), F12 = F13 =
    F23 = 0 are prescribed, P21, P22, P31, P32, P33 are zero."""
    return fix_rotation(*history_mixed_strain11(nsteps, 1.0 + lambda_end))


def history_case2(P_end, nsteps):
    """Case (2), full stress control: P-bar = P_end t / t_end (P_end: 9
    values, the final stress of case (1))."""
    t = np.arange(1, nsteps + 1)[:, None] / nsteps
    return np.ones((nsteps, 9), dtype=np.uint8), np.asarray(P_end, dtype=np.float64)[None, :] * t


def history_case3(F_end, nsteps):
    """Case (3), full strain control to the final F-bar of case (1), read as
    F-bar = I + (F_end - I) t / t_end (the printed F_end t / t_end would start
    from F = 0)."""
    eye = np.array([1.0, 0, 0, 0, 1.0, 0, 0, 0, 1.0])
    t = np.arange(1, nsteps + 1)[:, None] / nsteps
    return (np.zeros((nsteps, 9), dtype=np.uint8),
            eye[None, :] + (np.asarray(F_end, dtype=np.float64) - eye)[None, :] * t)


def history_case4(nsteps, lambda_end):
    """Case (4), the pseudo-uniaxial test of Sec. 3.2: full strain control
    F-bar = I + t/t_end diag(lambda_end, s, s), s = sqrt(1/(1 + lambda_end)) - 1
    (isochoric at the end in the transverse directions)."""
    s = np.sqrt(1.0 / (1.0 + lambda_end)) - 1.0
    d = np.array([lambda_end, 0, 0, 0, s, 0, 0, 0, s])
    eye = np.array([1.0, 0, 0, 0, 1.0, 0, 0, 0, 1.0])
    t = np.arange(1, nsteps + 1)[:, None] / nsteps
    return np.zeros((nsteps, 9), dtype=np.uint8), eye[None, :] + d[None, :] * t
