"""Observables of the two-component fields read back from a lattice: the
order parameter, the interface measure and the structure factor with the
domain size built from it (Sec. 5.3).  These are measurements of the output
(host arrays), not steps of the method.

* order parameter phi = (rho_A - rho_B) / (rho_A + rho_B) on fluid nodes,
  0 on particle nodes;
* interface measure A = sum over fluid nodes of (1 - phi^2) (it counts the
  sites inside the diffuse interfaces; the adjoint differentiates the same
  quantity);
* interface crossings: the lattice links (x, y and z neighbours, periodic)
  between two fluid nodes whose order parameters have opposite signs, a
  digital measure of the interface area (a flat interface normal to an axis
  crosses one link per site of its plane) that does not depend on the bulk
  densities of the phases;
* S(k) = < phi'(k) phi'(-k) >, phi' = phi - <phi>, averaged over spherical
  shells of width 2 pi / L in k = |k|, and the domain size
  L = 2 pi sum_k S(k) / sum_k k S(k) (Eq. 40 with the integrals as sums over
  the shells, k > 0).
"""
from __future__ import annotations

import math

import numpy as np


def order_parameter(rhoA: np.ndarray, rhoB: np.ndarray, owner: np.ndarray | None = None) -> np.ndarray:
    rt = rhoA + rhoB
    phi = np.zeros_like(rt)
    fluid = rt > 0 if owner is None else (owner < 0) & (rt > 0)
    phi[fluid] = (rhoA[fluid] - rhoB[fluid]) / rt[fluid]
    return phi


def interface_crossings(rhoA, rhoB, shape, owner=None) -> int:
    nx, ny, nz = shape
    phi = order_parameter(rhoA, rhoB, owner).reshape(nz, ny, nx)
    fluid = ((rhoA + rhoB > 0) if owner is None else (owner < 0)).reshape(nz, ny, nx)
    n = 0
    for ax in range(3):
        q = np.roll(phi, -1, axis=ax)
        both = fluid & np.roll(fluid, -1, axis=ax)
        n += int(np.count_nonzero(both & (phi * q < 0)))
    return n


def interface_measure(rhoA, rhoB, owner=None) -> float:
    phi = order_parameter(rhoA, rhoB, owner)
    fluid = (rhoA + rhoB > 0) if owner is None else (owner < 0)
    return float(np.sum(1.0 - phi[fluid] ** 2))


def structure_factor(phi: np.ndarray, shape) -> tuple:
    """(k, S(k)) averaged over spherical shells; phi in flat site order
    (x fastest)."""
    nx, ny, nz = shape
    f = phi.reshape(nz, ny, nx)
    f = f - f.mean()
    F = np.fft.fftn(f)
    S = (F * np.conj(F)).real / f.size
    kz = np.fft.fftfreq(nz) * 2 * math.pi
    ky = np.fft.fftfreq(ny) * 2 * math.pi
    kx = np.fft.fftfreq(nx) * 2 * math.pi
    K = np.sqrt(kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2)
    dk = 2 * math.pi / max(shape)
    shell = np.rint(K / dk).astype(int)
    nshell = shell.max() + 1
    sums = np.bincount(shell.ravel(), weights=S.ravel(), minlength=nshell)
    counts = np.bincount(shell.ravel(), minlength=nshell)
    k = np.arange(nshell) * dk
    Sk = np.where(counts > 0, sums / np.maximum(counts, 1), 0.0)
    return k[1:], Sk[1:]


def domain_size(k: np.ndarray, Sk: np.ndarray) -> float:
    """Eq. 40: L = 2 pi sum S / sum k S over the shells k > 0."""
    return float(2 * math.pi * np.sum(Sk) / np.sum(k * Sk))


def peak_wavenumber(k: np.ndarray, Sk: np.ndarray) -> float:
    return float(k[int(np.argmax(Sk))])
