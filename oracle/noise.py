"""CPU FP64 oracle for the noise-reduction step (Section V): brute-force sub-boxes and the
literal Lanczos (windowed-sinc) resampling sum.

TEST INFRASTRUCTURE ONLY -- see the package docstring.
"""
from __future__ import annotations

import math

import numpy as np

from . import core

# ----------------------------------------------------------------------------------------------
# method of sub-boxes (Section V A)
# ----------------------------------------------------------------------------------------------


def subbox_fields(model, disorder: str, mode: int) -> np.ndarray:
    """Per-atom amplitudes whose sub-box transforms are averaged, [model][site][n1][n2][n3][ncomp]:
    occupancy b delta (TOTAL) or b (delta - c) (DIFFUSE); moments M (TOTAL) or M - <M>
    (DIFFUSE).  The scattering length b is applied here, the form factor by the sum."""
    if disorder == "occ":
        x = model.occ.astype(np.float64)
        if mode == core.DIFFUSE:
            x = x - core.mean_occupancy(model)[None, :, None, None, None]
        x = x * model.scat_len[None, :, None, None, None]
        return x[..., None]
    if disorder == "spin":
        M = model.spins.astype(np.float64)
        if mode == core.DIFFUSE:
            M = M - core.mean_moment(model)[None, :, None, None, None, :]
        return M * model.scat_len[None, :, None, None, None, None]
    raise ValueError(disorder)


def all_origins(model) -> np.ndarray:
    """Every lattice point of every supercell, [(model, o1, o2, o3)] in C order."""
    grids = np.meshgrid(np.arange(model.nmodels), *(np.arange(c) for c in model.cells),
                        indexing="ij")
    return np.stack([g.reshape(-1) for g in grids], -1)


def subbox_intensity(model, disorder: str, mode: int, nsb: int, hkl: np.ndarray,
                     origins=None) -> np.ndarray:
    """Method of sub-boxes (Section V A).  Each origin (m, o) is the lattice point o of supercell
    m; its sub-box holds the atoms of the nsb^3 cells o + d, d in [0, nsb)^3, with open
    boundaries: at their unwrapped positions o + d + r_mu (+ u), with the data of the wrapped
    cells (o + d) mod n.  I(Q) = sum_origins |F_o(Q)|^2 / (norigin nsite nsb^3), magnetic
    C |F_o,perp|^2 (Eqs. mag_intensity, mag_projection).  origins=None: every lattice point of
    every supercell (the every-lattice-point variant); else rows (m, o1, o2, o3), e.g. drawn at
    random (the original random-origin variant).

    disorder "occ" / "spin": amplitudes of `subbox_fields`.  "disp": the atom at o + d + r_mu
    + u scatters with amplitude w = b delta (b without occupancies), exp(i Q.u) exact (no Taylor
    expansion); DIFFUSE subtracts from each atom the site mean of w cos(Q.u), i.e. b T_mu(Q)
    with `core.debye_waller(occupancy=True)`, so that nsb = n at a Bragg position of the
    supercell gives F - <F> of `core.displacive_intensity_direct`."""
    n = np.asarray(model.cells)
    d = np.stack(np.meshgrid(*(np.arange(nsb),) * 3, indexing="ij"), -1).reshape(-1, 3)
    nbox_atoms = d.shape[0] * model.nsite
    site = np.repeat(np.arange(model.nsite), d.shape[0])
    Q = core.q_cart(hkl, model.lattice)
    origins = all_origins(model) if origins is None else np.asarray(origins).reshape(-1, 4)
    if disorder == "disp":
        T = core.debye_waller(model, hkl, occupancy=True) if mode == core.DIFFUSE else None
    else:
        x = subbox_fields(model, disorder, mode)
        ncomp = x.shape[-1]
    acc = np.zeros(hkl.shape[0])
    for row in origins:
        m, o = int(row[0]), np.asarray(row[1:4])
        cells = o[None, :] + d                                       # unwrapped
        wrapped = np.mod(cells, n)
        frac = (cells[None, :, :] + model.sites[:, None, :]).reshape(-1, 3)
        if disorder == "disp":
            u = model.disp[m][:, wrapped[:, 0], wrapped[:, 1], wrapped[:, 2], :]
            u = u.reshape(nbox_atoms, 3).astype(np.float64)
            w = np.repeat(model.scat_len.astype(np.float64), d.shape[0])
            if model.occ is not None:
                w = w * model.occ[m][:, wrapped[:, 0], wrapped[:, 1], wrapped[:, 2]].reshape(-1)
            F = core.structure_factor(frac, u, w, site, model.ff_kind, model.ff_coef,
                                      model.lattice, hkl)[:, 0]
            if T is not None:
                for mu in range(model.nsite):
                    sel = site == mu
                    Fmu = core.structure_factor(frac[sel], None,
                                                np.full(d.shape[0], float(model.scat_len[mu])),
                                                site[sel], model.ff_kind, model.ff_coef,
                                                model.lattice, hkl)[:, 0]
                    F = F - T[:, mu] * Fmu
            acc += np.abs(F) ** 2
            continue
        amp = x[m][:, wrapped[:, 0], wrapped[:, 1], wrapped[:, 2], :].reshape(nbox_atoms, ncomp)
        F = core.structure_factor(frac, None, amp, site, model.ff_kind, model.ff_coef,
                                  model.lattice, hkl)
        if disorder == "spin":
            acc += core.perp_sq(F, Q)
        else:
            acc += np.abs(F[:, 0]) ** 2
    I = acc / (origins.shape[0] * model.nsite * nsb ** 3)
    return core.C_MAG * I if disorder == "spin" else I


# ----------------------------------------------------------------------------------------------
# Lanczos resampling (Section V B)
# ----------------------------------------------------------------------------------------------


def sinc(x):
    """sinc(x) = sin(x) / x, sinc(0) = 1 (the paper's unnormalised convention)."""
    x = np.asarray(x, dtype=np.float64)
    safe = np.where(x == 0.0, 1.0, x)
    return np.where(x == 0.0, 1.0, np.sin(safe) / safe)


def lanczos_parameters(m: int, mprime: int = 2):
    """(r_cut, m_eff): r_cut = 0.5 (1 - 1/m) for the plain window (m' = 2), and for the variant
    that reaches zero at 1/m', r_cut = (1 - 1/m)/m' with m replaced by m m'/2 in the window."""
    return (1.0 - 1.0 / m) / mprime, m * mprime / 2.0


def lanczos_weight(dQ: np.ndarray, m: int, mprime: int = 2) -> np.ndarray:
    """W(Q - G) = W_sinc(Q - G) L(Q - G) (Eqs. weight_sinc, windowed_sinc, lanczos), with
    dQ = Q - G in supercell-index units [..., 3]; strict window |dQ_alpha| < m_eff."""
    rcut, meff = lanczos_parameters(m, mprime)
    dQ = np.asarray(dQ, dtype=np.float64)
    wsinc = 8.0 * rcut ** 3 * np.prod(sinc(2.0 * math.pi * rcut * dQ), axis=-1)
    inside = np.all(np.abs(dQ) < meff, axis=-1)
    L = np.where(inside, np.prod(sinc(math.pi * dQ / meff), axis=-1), 0.0)
    return wsinc * L


def lanczos_support(Q: np.ndarray, m: int, mprime: int = 2) -> np.ndarray:
    """Integer offsets spanning [floor(Q) - m_eff + 1, floor(Q) + m_eff] per axis (the (2m)^3
    Bragg positions of Eq. lanczos), rounded outwards for a non-integer m_eff."""
    _, meff = lanczos_parameters(m, mprime)
    r = int(math.ceil(meff))
    off = np.arange(-r + 1, r + 1)
    return np.stack(np.meshgrid(off, off, off, indexing="ij"), -1).reshape(-1, 3)


def lanczos_resample(intensity_at_G, Q: np.ndarray, m: int, mprime: int = 2) -> np.ndarray:
    """I(Q) ~ sum_G I(G) W(Q - G) / sum_G W(Q - G) (Eq. intensity_convol_finite) for points Q
    in supercell-index units [nq, 3] (Q_alpha = n_alpha h_alpha, Eq. Q_def).

    `intensity_at_G(G)` returns I at integer supercell Bragg positions G [n, 3]."""
    Q = np.asarray(Q, dtype=np.float64)
    off = lanczos_support(Q, m, mprime)
    base = np.floor(Q).astype(np.int64)
    G = base[:, None, :] + off[None, :, :]                            # [nq, ntap, 3]
    W = lanczos_weight(Q[:, None, :] - G, m, mprime)                  # [nq, ntap]
    uniq, inv = np.unique(G.reshape(-1, 3), axis=0, return_inverse=True)
    IG = np.asarray(intensity_at_G(uniq), dtype=np.float64)[inv.reshape(-1)].reshape(W.shape)
    return np.sum(W * IG, axis=1) / np.sum(W, axis=1)


# ----------------------------------------------------------------------------------------------
# spherically symmetric cutoff (Section V B, the last of the three modifications)
# ----------------------------------------------------------------------------------------------


def inscribed_radius(model) -> float:
    """|r_max|: radius of the largest sphere inscribed in the supercell, half the smallest
    distance between opposite faces; the faces normal to a*_alpha are n_alpha 2 pi / |a*_alpha|
    apart."""
    B = core.reciprocal_vectors(model.lattice)
    return min(math.pi * n / float(np.linalg.norm(B[a])) for a, n in enumerate(model.cells))


def sphere_cutoff_radius(model, m: int, mprime: int = 2) -> float:
    """|r_c| = (1 - 1/m) |r_max|, scaled by 2/m' for the variant that decays to zero earlier
    (m' = 2 is the paper's expression)."""
    return (1.0 - 1.0 / m) * inscribed_radius(model) * 2.0 / mprime


def sphere_weight(qdist: np.ndarray, rc: float) -> np.ndarray:
    """W_r(|Q - G|) up to its constant prefactor: sin x / x^3 - cos x / x^2, x = |Q - G| |r_c|,
    with its limit 1/3 at x = 0 (series below x = 1e-3)."""
    x = np.asarray(qdist, dtype=np.float64) * rc
    small = np.abs(x) < 1e-3
    xs = np.where(small, 1.0, x)
    exact = np.sin(xs) / xs ** 3 - np.cos(xs) / xs ** 2
    return np.where(small, 1.0 / 3.0 - x * x / 30.0, exact)


def sphere_lanczos_weight(model, dQ: np.ndarray, m: int, mprime: int = 2) -> np.ndarray:
    """W = W_r(|Q - G|) L(Q - G): the spherical cutoff in place of Eq. weight_sinc, with the window
    L of Eq. lanczos (m replaced by m m'/2); dQ = Q - G in supercell-index units [..., 3]."""
    _, meff = lanczos_parameters(m, mprime)
    dQ = np.asarray(dQ, dtype=np.float64)
    n = np.asarray(model.cells, dtype=np.float64)
    dcart = (dQ / n) @ core.reciprocal_vectors(model.lattice)
    wr = sphere_weight(np.linalg.norm(dcart, axis=-1), sphere_cutoff_radius(model, m, mprime))
    inside = np.all(np.abs(dQ) < meff, axis=-1)
    L = np.where(inside, np.prod(sinc(math.pi * dQ / meff), axis=-1), 0.0)
    return wr * L


def sphere_resample(model, intensity_at_G, Q: np.ndarray, m: int, mprime: int = 2) -> np.ndarray:
    """Eq. intensity_convol_finite with W = W_r L over the same (2m)^3 Bragg positions as the
    separable window; Q in supercell-index units [nq, 3]."""
    Q = np.asarray(Q, dtype=np.float64)
    off = lanczos_support(Q, m, mprime)
    base = np.floor(Q).astype(np.int64)
    G = base[:, None, :] + off[None, :, :]
    W = sphere_lanczos_weight(model, Q[:, None, :] - G, m, mprime)
    uniq, inv = np.unique(G.reshape(-1, 3), axis=0, return_inverse=True)
    IG = np.asarray(intensity_at_G(uniq), dtype=np.float64)[inv.reshape(-1)].reshape(W.shape)
    return np.sum(W * IG, axis=1) / np.sum(W, axis=1)

