"""Seeded synthetic phase-space inputs: Philox4x64-10 uniforms + RAMBO momenta.

This module is the one piece shared by the CPU oracle's tests and the CUDA
path: it produces the momenta that both sides evaluate. It contains none of
the matrix-element arithmetic.

Counter-based stream (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random
numbers: as easy as 1, 2, 3"): Philox4x64 with 10 rounds, key = (seed, 0),
counter = (event index, particle slot, 0, 0).  Each block gives four 64-bit
words; a word w maps to the double u = ((w >> 11) + 0.5) * 2^-53, strictly
inside (0, 1), so log(u) is always finite.

Phase space: RAMBO (Kleiss, Stirling, Ellis, Comput. Phys. Commun. 40 (1986)
359): flat n-body massless phase space in the centre-of-mass frame at fixed
sqrt(s), followed by the standard rescaling of the 3-momenta that puts each
final state on its mass shell.  The paper's event generator samples momenta with MadEvent's
multichannel mapping (Sect. 2); that framework is not part of this project, so
flat RAMBO phase space stands in for it.

Layout: momenta[nevt][npar][4] float64, (E, px, py, pz) in GeV, initial
states first (p1 along +z, p2 along -z), then the final states in process
order.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "philox4x64_10",
    "uniforms",
    "rambo",
    "PROCESS_FINAL_MASSES",
    "process_momenta",
]

_M0 = np.uint64(0xD2E7470EE14C6C93)
_M1 = np.uint64(0xCA5A826395121157)
_W0 = np.uint64(0x9E3779B97F4A7C15)
_W1 = np.uint64(0xBB67AE8584CAA73B)
_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo64(a: np.ndarray, b: np.uint64):
    """Full 64x64 -> 128-bit product (hi, lo) of uint64 arrays, exact."""
    a_lo = a & _MASK32
    a_hi = a >> _S32
    b_lo = b & _MASK32
    b_hi = b >> _S32
    lo_lo = a_lo * b_lo
    hi_lo = a_hi * b_lo
    lo_hi = a_lo * b_hi
    hi_hi = a_hi * b_hi
    # cannot overflow: (2^32-1)^2 + 2*(2^32-1) = 2^64 - 1
    cross = (lo_lo >> _S32) + (hi_lo & _MASK32) + lo_hi
    hi = hi_hi + (hi_lo >> _S32) + (cross >> _S32)
    with np.errstate(over="ignore"):
        lo = a * b
    return hi, lo


def philox4x64_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox4x64-10 block function.

    ctr: uint64 array [..., 4]; key: uint64 array [..., 2] (broadcastable).
    Returns uint64 array [..., 4].
    """
    ctr = np.asarray(ctr, dtype=np.uint64)
    key = np.asarray(key, dtype=np.uint64)
    x0, x1, x2, x3 = (ctr[..., i].copy() for i in range(4))
    k0 = np.broadcast_to(key[..., 0], x0.shape).copy()
    k1 = np.broadcast_to(key[..., 1], x0.shape).copy()
    with np.errstate(over="ignore"):
        for r in range(10):
            hi0, lo0 = _mulhilo64(x0, _M0)
            hi1, lo1 = _mulhilo64(x2, _M1)
            x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
            if r != 9:
                k0 = k0 + _W0
                k1 = k1 + _W1
    return np.stack([x0, x1, x2, x3], axis=-1)


def uniforms(seed: int, first_event: int, nevt: int, nslots: int) -> np.ndarray:
    """Uniforms u[nevt][nslots][4] in (0,1) for events first_event..+nevt.

    Slot j of event i is the Philox block with counter (i, j, 0, 0) and key
    (seed, 0): event i's numbers never depend on how the batch was cut.
    """
    ev = np.arange(first_event, first_event + nevt, dtype=np.uint64)
    ctr = np.zeros((nevt, nslots, 4), dtype=np.uint64)
    ctr[:, :, 0] = ev[:, None]
    ctr[:, :, 1] = np.arange(nslots, dtype=np.uint64)[None, :]
    key = np.array([seed, 0], dtype=np.uint64)
    words = philox4x64_10(ctr, key)
    return ((words >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def rambo(sqrt_s: float, masses, u: np.ndarray) -> np.ndarray:
    """RAMBO final-state momenta [nevt][nfinal][4] from uniforms u[nevt][nfinal][4].

    Massless step: isotropic directions with energies drawn from q0 e^{-q0},
    then the conformal transformation (boost + scale) that takes the sum of
    the generated vectors to (sqrt_s, 0, 0, 0).  Mass-shell step: a common
    3-momentum scale xi, solved by Newton iteration, puts every final state on
    its mass shell while keeping total energy sqrt_s.
    """
    masses = np.asarray(masses, dtype=np.float64)
    nf = masses.shape[0]
    assert u.shape[1] == nf and u.shape[2] == 4
    c = 2.0 * u[..., 0] - 1.0
    s = np.sqrt(np.maximum(0.0, 1.0 - c * c))
    phi = 2.0 * np.pi * u[..., 1]
    q0 = -np.log(u[..., 2] * u[..., 3])
    q = np.stack([q0, q0 * s * np.cos(phi), q0 * s * np.sin(phi), q0 * c], axis=-1)
    Q = q.sum(axis=1)  # [nevt, 4]
    M = np.sqrt(Q[:, 0] ** 2 - (Q[:, 1:] ** 2).sum(axis=1))
    b = -Q[:, 1:] / M[:, None]
    gamma = Q[:, 0] / M
    a = 1.0 / (1.0 + gamma)
    x = sqrt_s / M
    bq = (b[:, None, :] * q[..., 1:]).sum(axis=2)  # [nevt, nf]
    p = np.empty_like(q)
    p[..., 0] = x[:, None] * (gamma[:, None] * q[..., 0] + bq)
    p[..., 1:] = x[:, None, None] * (
        q[..., 1:] + b[:, None, :] * q[..., 0:1] + a[:, None, None] * bq[..., None] * b[:, None, :]
    )
    # The conformal map leaves the 3-momentum sum and |E - |p|| at the rounding
    # level of its boost, which grows with the boost's gamma factor (up to
    # ~1e-12 relative).  The residual 3-momentum sum is removed evenly, and the
    # rescaling step below is applied in every case (for massless final
    # states it is a single exact step, xi = sqrt_s / sum |p|): it keeps the
    # zero sum and recomputes the energies from the 3-momenta, so the momenta
    # conserve 4-momentum and sit on their mass shells to rounding.
    p[..., 1:] -= p[..., 1:].sum(axis=1, keepdims=True) / nf
    if masses.sum() >= sqrt_s:
        raise ValueError("sqrt_s below the final-state mass threshold")
    p3sq = (p[..., 1:] ** 2).sum(axis=2)  # [nevt, nf]
    xi = np.full(p.shape[0], np.sqrt(1.0 - (masses.sum() / sqrt_s) ** 2))
    m2 = masses[None, :] ** 2
    for _ in range(60):
        e = np.sqrt(m2 + xi[:, None] ** 2 * p3sq)
        f = e.sum(axis=1) - sqrt_s
        df = (xi[:, None] * p3sq / e).sum(axis=1)
        step = f / df
        xi = xi - step
        if np.all(np.abs(step) <= 1e-16 * np.abs(xi)):
            break
    p[..., 1:] *= xi[:, None, None]
    p[..., 0] = np.sqrt(m2 + xi[:, None] ** 2 * p3sq)
    return p


# final-state masses per process, in the particle order of the process string
# (top mass is a parameter; placeholders "mt" are substituted by process_momenta)
PROCESS_FINAL_MASSES = {
    "e+ e- > mu+ mu-": (0.0, 0.0),
    "g g > t t~": ("mt", "mt"),
    "g g > t t~ g": ("mt", "mt", 0.0),
    "g g > t t~ g g": ("mt", "mt", 0.0, 0.0),
    "g g > t t~ g g g": ("mt", "mt", 0.0, 0.0, 0.0),
    "u u~ > t t~": ("mt", "mt"),
    "u u~ > t t~ g": ("mt", "mt", 0.0),
    "u u~ > t t~ g g": ("mt", "mt", 0.0, 0.0),
}


def process_momenta(proc: str, sqrt_s: float, nevt: int, seed: int,
                    first_event: int = 0, mt: float = 173.0) -> np.ndarray:
    """momenta[nevt][npar][4] for a process string at fixed sqrt(s)."""
    masses = [mt if m == "mt" else m for m in PROCESS_FINAL_MASSES[proc]]
    nf = len(masses)
    u = uniforms(seed, first_event, nevt, nf)
    pf = rambo(sqrt_s, masses, u)
    out = np.empty((nevt, nf + 2, 4), dtype=np.float64)
    e = 0.5 * sqrt_s
    out[:, 0] = (e, 0.0, 0.0, e)
    out[:, 1] = (e, 0.0, 0.0, -e)
    out[:, 2:] = pf
    return out
