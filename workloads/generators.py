"""Seeded input generators: ply layups, ply-angle noise and wrinkle fields.

All angles are in degrees, measured from the beam axis x toward y about +z.
Nothing here depends on the MS-GFEM method itself.
"""
import functools

import numpy as np

_CYCLE = (0.0, 90.0, 45.0, -45.0)


def layup_angles(n_plies: int, seed: int = 0) -> np.ndarray:
    """Symmetric layup built from the (0, 90, 45, -45) cycle.

    A half stack of floor(n/2) plies is read from the cycle starting at offset
    ``seed mod 4``; an odd stack gets one middle ply (the next cycle entry); the
    half stack is then mirrored.  For 8 plies and seed 0 this is [0/90/45/-45]s.
    Index 0 is the bottom ply (z = 0).
    """
    if n_plies <= 0:
        raise ValueError("n_plies must be positive")
    off = seed % 4
    half = [_CYCLE[(off + i) % 4] for i in range(n_plies // 2)]
    mid = [_CYCLE[(off + n_plies // 2) % 4]] if n_plies % 2 else []
    return np.array(half + mid + half[::-1], dtype=np.float64)


def ply_angles(cfg) -> np.ndarray:
    """Per-ply angles of a beam workload: layup plus optional Gaussian noise."""
    ang = layup_angles(cfg.NZ, cfg.layup_seed)
    if cfg.noise_sd_deg > 0.0:
        rng = np.random.default_rng(cfg.noise_seed)
        ang = ang + cfg.noise_sd_deg * rng.standard_normal(cfg.NZ)
    return ang


@functools.lru_cache(maxsize=8)
def _wrinkle_factor(NX, NY, NZ, hx, hy, t, sd_deg, corr_len):
    xs = (np.arange(NX) + 0.5) * hx
    ys = (np.arange(NY) + 0.5) * hy
    zs = (np.arange(NZ) + 0.5) * t
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    d2 = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    cov = sd_deg ** 2 * np.exp(-d2 / (2.0 * corr_len ** 2))
    cov[np.diag_indices_from(cov)] += 1e-10 * sd_deg ** 2
    L = np.linalg.cholesky(cov)
    L.setflags(write=False)
    return L


def wrinkle_field(cfg, sample: int, sd_deg: float = 3.0, corr_len: float = 10.0) -> np.ndarray:
    """Gaussian random field of ply-angle perturbation at element centroids.

    Squared-exponential covariance sd^2 exp(-|x - x'|^2 / (2 l^2)) in 3-D,
    sampled through a Cholesky factor of the covariance with a jitter of
    1e-10 sd^2 on the diagonal (computed once per mesh); the sample index is
    the seed.  Returns an array of shape (NX, NY, NZ) in degrees.
    """
    L = _wrinkle_factor(cfg.NX, cfg.NY, cfg.NZ, cfg.hx, cfg.hy, cfg.t, float(sd_deg), float(corr_len))
    rng = np.random.default_rng(sample)
    return (L @ rng.standard_normal(L.shape[0])).reshape(cfg.NX, cfg.NY, cfg.NZ)


def element_angles(cfg, sample=None) -> np.ndarray:
    """Per-element fibre angle, shape (NX, NY, NZ): ply angle of layer k, plus
    the wrinkle field of ``sample`` when one is given."""
    ang = np.broadcast_to(ply_angles(cfg)[None, None, :], (cfg.NX, cfg.NY, cfg.NZ)).copy()
    if sample is not None:
        ang += wrinkle_field(cfg, sample)
    return ang
