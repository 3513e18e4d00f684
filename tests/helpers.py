"""Shared helpers of the GPU parity tests (inputs, oracle geometry, error norms)."""
import numpy as np

from paper_2309_01977_gb300 import phantom


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def max_abs_rel(a, b) -> float:
    """max |a - b| over max |b|: an error localised in one tile or strip is
    not diluted by the rest of the array, as it is in the relative L2."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def assert_close(got, ref, tol, what=""):
    """Relative L2 within tol, and every element within 10 tol of max |ref|."""
    e2, einf = rel_l2(got, ref), max_abs_rel(got, ref)
    assert e2 <= tol, (what, "rel L2", e2)
    assert einf <= 10 * tol, (what, "max abs / max |ref|", einf)


def f32(a) -> np.ndarray:
    """Round to float32 and back, so that the oracle sees exactly the GPU's inputs."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def oracle_geom(oracle, g, mu64):
    """Oracle geometry equal to the library Geometry g (same float32 parameters)."""
    return oracle.Geom(n=g.n, nz=g.nz, n_angles=g.n_angles, angles=g.angles_rad,
                       voxel_cm=float(np.float32(g.voxel_cm)), mu=mu64 if g.attenuation else None,
                       use_psf=g.psf, sigma0=float(np.float32(g.psf_sigma0)),
                       slope=float(np.float32(g.psf_slope)), nsigma=float(np.float32(g.psf_nsigma)),
                       det_offset=float(np.float32(g.det_offset)),
                       det_offsets=None if g.det_offsets is None else [float(np.float32(v)) for v in g.det_offsets],
                       trans=None if g.det_shifts is None else [float(np.float32(v)) for v in g.det_shifts],
                       fov=None if g.fov_mask is None else f32(g.fov_mask))


def phantom_inputs(n, nz, seed):
    f, mu = phantom.make_phantom(n, nz, seed)
    return f32(f), f32(mu)


def one_hot_projection(oracle, og, voxel, rmax):
    """H e_v of the oracle for the unit volume at `voxel` = (i, j, k), from the
    z slab the voxel's blur reaches: rotation and attenuation act on every z
    plane alone and the PSF spreads at most rmax bins along z, so the
    projection of e_v is zero outside [k - rmax, k + rmax] and, inside, equals
    the projection of the slab [k - rmax - 1, k + rmax + 2) cut from the
    volume and the mu map (edges of the real volume stay where they are).
    Returns the full [n_angles][n][nz] array."""
    import dataclasses
    i, j, k = voxel
    zlo, zhi = max(0, k - rmax - 1), min(og.nz, k + rmax + 2)
    e = np.zeros((og.n, og.n, zhi - zlo))
    e[i, j, k - zlo] = 1.0
    og_c = dataclasses.replace(og, nz=zhi - zlo, mu=None if og.mu is None else np.asarray(og.mu)[:, :, zlo:zhi])
    c = np.zeros((og.n_angles, og.n, og.nz))
    c[:, :, zlo:zhi] = oracle.forward(e, og_c)
    return c
