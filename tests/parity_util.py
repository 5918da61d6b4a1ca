"""Comparison helpers of the GPU parity tests (no GPU code here).

Eigenvalues are compared one by one: a non-rigid eigenvalue relative to
itself, |lambda_gpu - lambda_oracle| <= tol |lambda_oracle|, and the rigid-body
zeros of floating subdomains (Sec. 5.2: exact zero eigenvalues) absolutely at
tol times the largest eigenvalue given (at least 1).  Solutions are compared in the
energy norm ||v||_a = sqrt(v^T A v) of the oracle's assembled matrix.
"""
import numpy as np


def _scale(ref):
    # the largest eigenvalue given (the oracle may give one beyond the wanted
    # ones), at least 1: the eigenvalues are ratios of energies, so a subdomain
    # whose wanted pairs are all rigid zeros is compared at the scale 1
    return max(float(np.abs(np.asarray(ref, dtype=np.float64)).max()), 1.0)


def rigid_mask(ref):
    """Oracle eigenvalues that are rigid-body zeros (below 1e-8 of the scale)."""
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(ref) <= 1e-8 * _scale(ref)


def eig_errors(lam, ref):
    """(largest relative error of the non-rigid eigenvalues, largest rigid
    eigenvalue divided by the scale).  ``ref`` may hold more eigenvalues than
    ``lam`` (they set the scale only)."""
    lam = np.asarray(lam, dtype=np.float64)
    full = np.asarray(ref, dtype=np.float64)
    ref = full[:lam.size]
    rig = np.abs(ref) <= 1e-8 * _scale(full)
    rel = np.abs(lam - ref)[~rig] / np.abs(ref[~rig]) if np.any(~rig) else np.zeros(1)
    zero = np.abs(lam[rig]) / _scale(full) if np.any(rig) else np.zeros(1)
    return float(rel.max()), float(zero.max())


def assert_eigs(lam, ref, tol, what=""):
    rel, zero = eig_errors(lam, ref)
    assert rel <= tol and zero <= tol, (what, rel, zero, np.asarray(lam), np.asarray(ref))
    return rel, zero


def energy_rel(A, x, y):
    """||x - y||_a / ||y||_a."""
    d = np.asarray(x, dtype=np.float64) - np.asarray(y, dtype=np.float64)
    den = float(y @ (A @ y))
    return float(np.sqrt(max(float(d @ (A @ d)), 0.0) / den)) if den > 0 else float(np.sqrt(max(float(d @ (A @ d)), 0.0)))


def energy_error_direct(A, b, uh_energy_sq, u):
    """||u_h - u||_a / ||u_h||_a for any u, from A u_h = b:
    ||u_h - u||_a^2 = ||u_h||_a^2 - 2 b^T u + u^T A u."""
    e2 = uh_energy_sq - 2.0 * float(b @ u) + float(u @ (A @ u))
    return float(np.sqrt(max(e2, 0.0) / uh_energy_sq))
