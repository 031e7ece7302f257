"""CPU FP64 oracle: geometry, the direct Fourier sum (part 1) and the FFT method (part 2).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

Notation follows the paper (arXiv 1809.07088):
  * supercell of n1 n2 n3 unit cells, lattice points R, sites mu at fractional r_mu (Eq. r_vec);
  * supercell Bragg positions G = (G1/n1) a* + (G2/n2) b* + (G3/n3) c*, G_alpha integer
    (Eq. G_def), split as G = H + k with k_alpha = G_alpha mod n_alpha (Eq. g_vec);
  * a* = 2 pi b x c / V etc. (Section II).
Grids are passed either as r.l.u. points `hkl` [nq, 3] (direct sum, any Q) or as integer
supercell indices `G` [nvox, 3] (FFT method, commensurate grid only).
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import build as _build

TWO_PI = 2.0 * math.pi
C_MAG = 0.07265  # barn; magnetic constant (gamma_n r_0 / 2)^2 of Eq. mag_intensity
TOTAL, DIFFUSE = 0, 1

# ----------------------------------------------------------------------------------------------
# geometry and form factors
# ----------------------------------------------------------------------------------------------


def lattice_vectors(lattice) -> np.ndarray:
    """Rows a, b, c in Cartesian Angstrom: a along x, b in the xy plane (standard setting)."""
    a, b, c, al, be, ga = lattice
    al, be, ga = (math.radians(x) for x in (al, be, ga))
    va = np.array([a, 0.0, 0.0])
    vb = np.array([b * math.cos(ga), b * math.sin(ga), 0.0])
    cx = c * math.cos(be)
    cy = c * (math.cos(al) - math.cos(be) * math.cos(ga)) / math.sin(ga)
    cz = math.sqrt(c * c - cx * cx - cy * cy)
    return np.array([va, vb, [cx, cy, cz]])


def reciprocal_vectors(lattice) -> np.ndarray:
    """Rows a*, b*, c* with a* = 2 pi (b x c) / V, V = a . (b x c) (Section II)."""
    va, vb, vc = lattice_vectors(lattice)
    vol = float(np.dot(va, np.cross(vb, vc)))
    return TWO_PI * np.array([np.cross(vb, vc), np.cross(vc, va), np.cross(va, vb)]) / vol


def q_cart(hkl: np.ndarray, lattice) -> np.ndarray:
    """Q = h a* + k b* + l c* (Eq. Q_def), Cartesian 1/A."""
    return np.asarray(hkl, dtype=np.float64) @ reciprocal_vectors(lattice)


def form_factor(kind: int, coef, qnorm: np.ndarray) -> np.ndarray:
    """kind 0: 1; kind 1: sum_i a_i exp(-b_i s^2) + c; kind 2: <j0>; s = |Q| / 4 pi."""
    s2 = (np.asarray(qnorm, dtype=np.float64) / (4.0 * math.pi)) ** 2
    c = np.asarray(coef, dtype=np.float64)
    if kind == 1:
        return (c[0] * np.exp(-c[4] * s2) + c[1] * np.exp(-c[5] * s2) +
                c[2] * np.exp(-c[6] * s2) + c[3] * np.exp(-c[7] * s2) + c[8])
    if kind == 2:
        return c[0] * np.exp(-c[1] * s2) + c[2] * np.exp(-c[3] * s2) + c[4] * np.exp(-c[5] * s2) + c[6]
    return np.ones_like(s2)


def site_form_factors(model, qnorm: np.ndarray) -> np.ndarray:
    """[nq, nsite] form factors times scattering lengths b_mu f_mu(|Q|)."""
    out = np.empty((qnorm.shape[0], model.nsite))
    for s in range(model.nsite):
        out[:, s] = model.scat_len[s] * form_factor(int(model.ff_kind[s]), model.ff_coef[s], qnorm)
    return out


def is_integer_hkl(hkl: np.ndarray, tol=1e-9) -> np.ndarray:
    return np.all(np.abs(hkl - np.rint(hkl)) < tol, axis=1)


# ----------------------------------------------------------------------------------------------
# part 1: direct Fourier sum (the C loop in direct.c)
# ----------------------------------------------------------------------------------------------

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_structure_factor.argtypes = [ctypes.c_long, dp, dp, ctypes.c_int, dp, ip,
                                                ctypes.c_int, ip, dp, dp, ctypes.c_long, dp, dp]
        lib.oracle_structure_factor.restype = None
        lib.oracle_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def oracle_threads() -> int:
    return int(_load().oracle_threads())


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def structure_factor(frac, ucart, amp, site, ff_kind, ff_coef, lattice, hkl) -> np.ndarray:
    """F(Q) = sum_j amp_j f_j(|Q|) exp(i Q . r_j), Eq. sf, for every row of `hkl`.

    frac [natom, 3]: R + r_mu in fractional cell coordinates; ucart [natom, 3] Cartesian
    displacement or None; amp [natom, ncomp] (ncomp <= 3).  Returns complex [nq, ncomp]."""
    lib = _load()
    frac = np.ascontiguousarray(frac, dtype=np.float64)
    amp = np.ascontiguousarray(amp, dtype=np.float64)
    if amp.ndim == 1:
        amp = amp[:, None]
    natom, ncomp = amp.shape
    assert ncomp <= 3 and frac.shape == (natom, 3)
    site = np.ascontiguousarray(site, dtype=np.int32)
    kinds = np.ascontiguousarray(ff_kind, dtype=np.int32)
    coef = np.ascontiguousarray(ff_coef, dtype=np.float64).reshape(-1, 9)
    recip = np.ascontiguousarray(reciprocal_vectors(lattice))
    hkl = np.ascontiguousarray(hkl, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((hkl.shape[0], ncomp, 2))
    u = None
    if ucart is not None:
        u = np.ascontiguousarray(ucart, dtype=np.float64)
        assert u.shape == (natom, 3)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.oracle_structure_factor(natom, _dp(frac), _dp(u) if u is not None else None, ncomp,
                                _dp(amp), site.ctypes.data_as(ip), len(kinds),
                                kinds.ctypes.data_as(ip), _dp(coef), _dp(recip), hkl.shape[0],
                                _dp(hkl), _dp(out))
    return out[..., 0] + 1j * out[..., 1]


def atom_list(model):
    """(frac [natom, 3], site [natom]) with atoms ordered [site][R1][R2][R3] like the arrays."""
    n1, n2, n3 = model.cells
    R = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1)
    frac = R[None].astype(np.float64) + model.sites[:, None, None, None, :]
    site = np.repeat(np.arange(model.nsite), model.ncell)
    return frac.reshape(-1, 3), site


def mean_occupancy(model) -> np.ndarray:
    """c_mu: given, else the sample mean over lattice points and supercells (Eq. occ)."""
    if model.mean_occ is not None:
        return np.asarray(model.mean_occ, dtype=np.float64)
    return model.occ.astype(np.float64).mean(axis=(0, 2, 3, 4))


def mean_moment(model) -> np.ndarray:
    return model.spins.astype(np.float64).mean(axis=(0, 2, 3, 4))  # [nsite, 3]


def _sf(model, frac, u, amp, site, hkl):
    return structure_factor(frac, u, amp, site, model.ff_kind, model.ff_coef, model.lattice, hkl)


def _cell_sf(model, amp_per_site, hkl):
    """sum_mu amp_mu b_mu f_mu exp(i G . r_mu): one atom per site at r_mu."""
    return _sf(model, model.sites, None, amp_per_site, np.arange(model.nsite), hkl)


def occupancy_bragg(model, hkl) -> np.ndarray:
    """<F_c(G)> = n1 n2 n3 delta_{G,H} sum_mu c_mu b_mu exp(i G . r_mu): Eq. bragg_sf, T = 1."""
    c = mean_occupancy(model)
    amp = model.ncell * c * model.scat_len
    Fb = _cell_sf(model, amp[:, None], hkl)[:, 0]
    return np.where(is_integer_hkl(hkl), Fb, 0.0)


def occupancy_intensity_direct(model, hkl, mode=DIFFUSE) -> np.ndarray:
    """I = (1/N) < |F - <F>|^2 > (Eqs. intensity_sf, sf, bragg_diffuse_sf), F from the occupied
    atoms (amplitude b delta), averaged over the supercells of the ensemble; TOTAL: no <F>."""
    frac, site = atom_list(model)
    bragg = occupancy_bragg(model, hkl) if mode == DIFFUSE else 0.0
    acc = np.zeros(hkl.shape[0])
    for m in range(model.nmodels):
        amp = model.scat_len[site] * model.occ[m].reshape(-1).astype(np.float64)
        F = _sf(model, frac, None, amp, site, hkl)[:, 0] - bragg
        acc += np.abs(F) ** 2
    return acc / (model.nmodels * model.natom)


def displacive_weights(model, m) -> np.ndarray:
    """w = b delta (occupancy given) or b: per-atom amplitude of the displacive model."""
    _, site = atom_list(model)
    w = model.scat_len[site].astype(np.float64)
    if model.occ is not None:
        w = w * model.occ[m].reshape(-1)
    return w


def displacive_bragg(model, hkl) -> np.ndarray:
    """<F(H)> of Eq. bragg_sf_disp: only the even Taylor orders survive, i.e. the even part
    (F(u) + F(-u)) / 2 = sum b f e^{iH.(R+r)} cos(H.u) at integer H, averaged over supercells."""
    frac, site = atom_list(model)
    integer = is_integer_hkl(hkl)
    out = np.zeros(hkl.shape[0], dtype=np.complex128)
    if not integer.any():
        return out
    hi = hkl[integer]
    acc = np.zeros(hi.shape[0], dtype=np.complex128)
    for m in range(model.nmodels):
        u = model.disp[m].reshape(-1, 3).astype(np.float64)
        w = displacive_weights(model, m)
        acc += 0.5 * (_sf(model, frac, u, w, site, hi)[:, 0] + _sf(model, frac, -u, w, site, hi)[:, 0])
    out[integer] = acc / model.nmodels
    return out


def displacive_intensity_direct(model, hkl, mode=DIFFUSE, return_F=False):
    """I = (1/N) < |F - <F>|^2 > with F = sum_j w_j f_j exp(i Q.(R + r_mu + u_j)) (Eq. sf with
    Eq. r_vec), <F> from `displacive_bragg` in DIFFUSE mode (Eq. disp_diffuse_intensity)."""
    frac, site = atom_list(model)
    bragg = displacive_bragg(model, hkl) if mode == DIFFUSE else 0.0
    acc = np.zeros(hkl.shape[0])
    Fs = []
    for m in range(model.nmodels):
        u = model.disp[m].reshape(-1, 3).astype(np.float64)
        F = _sf(model, frac, u, displacive_weights(model, m), site, hkl)[:, 0] - bragg
        acc += np.abs(F) ** 2
        Fs.append(F)
    I = acc / (model.nmodels * model.natom)
    return (I, np.array(Fs)) if return_F else I


def perp_sq(F: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """|F_perp|^2 for F_perp = G^ x F x G^ (Eq. mag_projection) = |F|^2 - |G^ . F|^2.
    At Q = 0 the direction is undefined; the orientational average (2/3)|F|^2 is returned."""
    qn = np.linalg.norm(Q, axis=1)
    tot = np.sum(np.abs(F) ** 2, axis=1)
    safe = np.where(qn > 0, qn, 1.0)
    qhat = Q / safe[:, None]
    par = np.abs(np.sum(qhat * F, axis=1)) ** 2
    return np.where(qn > 0, tot - par, (2.0 / 3.0) * tot)


def debye_waller(model, hkl, occupancy=False, chunk=2048) -> np.ndarray:
    """T_mu(Q) of Eq. dw for every row of `hkl` and every site, [nq, nsite]: the mean over the
    lattice points R and the supercells of (1 + a) exp(i Q.u_R,mu).  The odd orders of Q.u
    average to zero over the ensemble (Section III C), so the even part, the mean of
    (1 + a) cos(Q.u), is kept: the same reading as <F(H)> in `displacive_bragg`.  With
    occupancy=True the weight 1 + a is the occupancy delta of each atom (when the model has
    occupancies); otherwise it is 1 (the moments of the magnetic case carry their own size)."""
    Q = q_cart(hkl, model.lattice)
    out = np.zeros((Q.shape[0], model.nsite))
    for mu in range(model.nsite):
        u = model.disp[:, mu].reshape(-1, 3).astype(np.float64)          # [(model, R), 3]
        w = np.ones(u.shape[0])
        if occupancy and model.occ is not None:
            w = model.occ[:, mu].reshape(-1).astype(np.float64)
        for q0 in range(0, Q.shape[0], chunk):
            out[q0:q0 + chunk, mu] = np.cos(Q[q0:q0 + chunk] @ u.T) @ w / u.shape[0]
    return out


def magnetic_intensity_direct(model, hkl, mode=TOTAL, dw=False) -> np.ndarray:
    """I_mag = (C/N) < |F_perp|^2 >, F_mag = sum f_mag T_mu M_j exp(i G.r_j) (Eqs. mag_sf,
    mag_intensity, mag_projection), T_mu = 1, or with dw=True the Debye-Waller factor of the
    model's displacements (`debye_waller`), the only coupling of the moments to the
    displacements in Eq. mag_sf.  DIFFUSE subtracts the structure factor of the mean moment of
    each site (zero when the moments have no long-range order)."""
    frac, site = atom_list(model)
    Q = q_cart(hkl, model.lattice)
    integer = is_integer_hkl(hkl)[:, None]
    mbar = mean_moment(model) * model.ncell * model.scat_len[:, None]
    T = debye_waller(model, hkl) if dw else None
    acc = np.zeros(hkl.shape[0])
    for m in range(model.nmodels):
        amp = model.spins[m].reshape(-1, 3).astype(np.float64) * model.scat_len[site][:, None]
        if T is None:
            F = _sf(model, frac, None, amp, site, hkl)
            if mode == DIFFUSE:
                F = F - _cell_sf(model, mbar, hkl) * integer
        else:
            F = np.zeros((hkl.shape[0], 3), dtype=np.complex128)
            for mu in range(model.nsite):
                sel = site == mu
                Fmu = _sf(model, frac[sel], None, amp[sel], site[sel], hkl)
                if mode == DIFFUSE:
                    Fmu = Fmu - _sf(model, model.sites[mu:mu + 1], None, mbar[mu:mu + 1],
                                    np.array([mu]), hkl) * integer
                F += T[:, mu, None] * Fmu
        acc += perp_sq(F, Q)
    return C_MAG * acc / (model.nmodels * model.natom)


# ----------------------------------------------------------------------------------------------
# part 2: the FFT method, step by step (Section III)
# ----------------------------------------------------------------------------------------------


def lattice_fft(x: np.ndarray) -> np.ndarray:
    """X_k = sum_R x_R exp(+2 pi i sum_alpha k_alpha R_alpha / n_alpha) over the last three
    axes (Eq. fft with N_alpha = n_alpha), unnormalised.  numpy's inverse FFT carries the +i
    sign and a 1/(n1 n2 n3) factor, which is undone here."""
    n = x.shape[-1] * x.shape[-2] * x.shape[-3]
    return np.fft.ifftn(x, axes=(-3, -2, -1)) * n


def split_G(G: np.ndarray, cells) -> np.ndarray:
    """k of G = H + k (Eq. g_vec): k_alpha = G_alpha mod n_alpha."""
    return np.mod(G, np.asarray(cells, dtype=np.int64))


def site_phases(model, G: np.ndarray) -> np.ndarray:
    """exp(i G . r_mu) = exp(2 pi i sum_alpha (G_alpha / n_alpha) r_mu,alpha): [nvox, nsite]."""
    hkl = G / np.asarray(model.cells, dtype=np.float64)
    t = hkl @ model.sites.T
    t = t - np.floor(t)
    return np.exp(1j * TWO_PI * t)


def _phi(model, G):
    """phi_mu(G) = b_mu f_mu(|G|) exp(i G.r_mu), with the Cartesian Q of every voxel."""
    hkl = G / np.asarray(model.cells, dtype=np.float64)
    Q = q_cart(hkl, model.lattice)
    ff = site_form_factors(model, np.linalg.norm(Q, axis=1))
    return ff * site_phases(model, G), Q


def occupancy_intensity_fft(model, G, mode=DIFFUSE) -> np.ndarray:
    """Eqs. occ, comp_sf_diffuse, comp_ft, comp_diffuse_intensity.

    DIFFUSE: x_R = delta_R - c_mu (= c a_R of Eq. occ) is transformed, so that
    F_c - <F_c> = sum_mu a_k c b exp(iG.r_mu); TOTAL: x_R = delta_R."""
    occ = model.occ.astype(np.float64)
    if mode == DIFFUSE:
        occ = occ - mean_occupancy(model)[None, :, None, None, None]
    X = lattice_fft(occ)                                  # [model][site][k1][k2][k3]
    k = split_G(G, model.cells)
    phi, _ = _phi(model, G)                               # b f exp(iG.r) per voxel and site
    Xk = X[:, :, k[:, 0], k[:, 1], k[:, 2]]               # [model][site][nvox]
    F = np.einsum("vs,msv->mv", phi, Xk)
    return np.mean(np.abs(F) ** 2, axis=0) / model.natom


def magnetic_intensity_fft(model, G, mode=TOTAL, dw=False) -> np.ndarray:
    """Eqs. mag_sf (T = 1, or with dw=True the Debye-Waller factor of Eq. dw from
    `debye_waller`), mag_ft (one FFT per Cartesian component), mag_intensity, mag_projection."""
    M = model.spins.astype(np.float64)                    # [model][site][n1][n2][n3][3]
    if mode == DIFFUSE:
        M = M - mean_moment(model)[None, :, None, None, None, :]
    X = lattice_fft(np.moveaxis(M, -1, 2))                # [model][site][3][k1][k2][k3]
    k = split_G(G, model.cells)
    phi, Q = _phi(model, G)
    if dw:
        phi = phi * debye_waller(model, G / np.asarray(model.cells, dtype=np.float64))
    Xk = X[:, :, :, k[:, 0], k[:, 1], k[:, 2]]            # [model][site][3][nvox]
    acc = np.zeros(G.shape[0])
    for m in range(model.nmodels):
        F = np.einsum("vs,sav->va", phi, Xk[m])
        acc += perp_sq(F, Q)
    return C_MAG * acc / (model.nmodels * model.natom)


def monomials(P: int):
    """Exponent triples (a, b, c) with a + b + c = n <= P, graded by n, then a, b descending:
    the distinct monomials u_x^a u_y^b u_z^c of Eq. gu_expansion; order n has (n+1)(n+2)/2."""
    out = []
    for n in range(P + 1):
        for a in range(n, -1, -1):
            for b in range(n - a, -1, -1):
                out.append((a, b, n - a - b))
    return out


def x_max(model, qgrid) -> float:
    """max |Q . u| over all atoms and all Q of the requested box: Q . u is linear in Q, so the
    maximum over the parallelepiped is reached at one of its 8 corners."""
    corners = []
    for i in (0, qgrid.count[0] - 1):
        for j in (0, qgrid.count[1] - 1):
            for l in (0, qgrid.count[2] - 1):
                corners.append([qgrid.h0[0] + i * qgrid.step[0], qgrid.h0[1] + j * qgrid.step[1],
                                qgrid.h0[2] + l * qgrid.step[2]])
    Qc = q_cart(np.array(corners), model.lattice)         # [8, 3]
    u = model.disp.reshape(-1, 3).astype(np.float64)
    return float(np.max(np.abs(u @ Qc.T)))


def taylor_order(xmax: float, eps: float) -> int:
    """Smallest order P with remainder bound x^(P+1)/(P+1)! <= eps (Section III C)."""
    P = 0
    while (P + 1) * math.log(max(xmax, 1e-300)) - math.lgamma(P + 2) > math.log(eps):
        P += 1
        if P > 200:
            raise ValueError("Taylor order above 200")
    return P


def zone_taylor_orders(model, qgrid, eps: float, G=None):
    """Taylor order per voxel under the per-zone reading of the remainder bound of Section
    III C, and the single order P of the whole grid.

    A zone is the set of grid voxels G = n H + k sharing one H = floor(G / n).  By
    Cauchy-Schwarz |Q . u_j| <= |Q| |u_j|, so over a zone max_j |Q . u_j| <= x_H =
    min(q_H u_max, x_max), with q_H the largest |Q| over the zone's voxels (|Q| is convex, so it
    is reached at a corner of the zone's box of voxels) and u_max the largest |u_j| of the
    ensemble.  The zone's order is the smallest order whose bound x_H^(P+1)/(P+1)! <= eps,
    never above P.  Returns (orders, P): orders [nvox] for every voxel of the grid, or for the
    voxels G [nq, 3] (supercell indices inside the grid) when given."""
    n = np.asarray(model.cells, dtype=np.int64)
    glo = np.rint(np.asarray(qgrid.h0) * n).astype(np.int64)
    ghi = glo + np.asarray(qgrid.count, dtype=np.int64) - 1
    xm = x_max(model, qgrid)
    P = taylor_order(xm, eps)
    u = model.disp.reshape(-1, 3).astype(np.float64)
    umax = float(np.max(np.sqrt(np.sum(u * u, axis=1))))
    Hlo, Hhi = np.floor_divide(glo, n), np.floor_divide(ghi, n)
    nH = Hhi - Hlo + 1
    table = np.empty(tuple(nH), dtype=np.int64)
    for h in np.ndindex(*table.shape):
        Hz = Hlo + np.array(h)
        lo = np.maximum(n * Hz, glo)
        hi = np.minimum(n * Hz + n - 1, ghi)
        box = np.array([[(hi if (c >> (2 - a)) & 1 else lo)[a] for a in range(3)] for c in range(8)])
        qmax = float(np.max(np.linalg.norm(q_cart(box / n[None, :], model.lattice), axis=1)))
        table[h] = min(P, taylor_order(min(qmax * umax, xm), eps))
    if G is None:
        G = qgrid.g_index(model.cells)
    h = np.floor_divide(np.asarray(G, dtype=np.int64), n[None, :]) - Hlo[None, :]
    return table[h[:, 0], h[:, 1], h[:, 2]], P


def displacive_intensity_fft(model, G, mode=DIFFUSE, P=None, eps=1e-8, return_F=False, P_vox=None):
    """Taylor-expanded FFT method, Eqs. disp_expansion, gu_expansion, total_sf_taylor, U_fft,
    A_fft, bragg_sf_disp, disp_diffuse_intensity.

    For each site and each distinct monomial t = (a, b, c) of order n = a + b + c <= P the field
    w_R u_x^a u_y^b u_z^c (w = b delta, i.e. c b (1 + a_R) of Eq. A_fft, or b) is transformed by
    `lattice_fft`; the orderings alpha(n) of Eq. gu_expansion that give the same monomial
    collapse into the multinomial weight n!/(a! b! c!), so the term's coefficient is
    i^n Q_x^a Q_y^b Q_z^c / (a! b! c!) with Q Cartesian and u in Angstrom.  The Bragg term keeps
    the even orders of the k = 0 transforms averaged over the supercells.  Streaming over
    monomials keeps the memory at one field at a time.  P_vox (optional, [nvox]): the order of
    each voxel (zone orders); each voxel then keeps only its monomials of order n <= P_vox, the
    Bragg term included; P must be at least max(P_vox)."""
    if P is None:
        raise ValueError("pass the Taylor order P")
    keep_n = None if P_vox is None else np.asarray(P_vox)[None, :] >= np.arange(P + 1)[:, None]  # [n][nvox]
    k = split_G(G, model.cells)
    phi, Q = _phi(model, G)
    nv = G.shape[0]
    pw = [Q[:, a][:, None] ** np.arange(P + 1)[None, :] for a in range(3)]   # [nvox, P+1]
    bragg_vox = np.all(k == 0, axis=1)
    u = model.disp.astype(np.float64)                     # [model][site][n1][n2][n3][3]
    F = np.zeros((model.nmodels, nv), dtype=np.complex128)
    Fb = np.zeros(nv, dtype=np.complex128)
    for mu in range(model.nsite):
        # b_mu sits in phi; the field weight is the occupancy (or 1)
        w = np.ones((model.nmodels,) + tuple(model.cells))
        if model.occ is not None:
            w = w * model.occ[:, mu]
        S = np.zeros((model.nmodels, nv), dtype=np.complex128)
        Sb = np.zeros(nv, dtype=np.complex128)
        ux, uy, uz = u[:, mu, ..., 0], u[:, mu, ..., 1], u[:, mu, ..., 2]
        for (a, b, c) in monomials(P):
            n = a + b + c
            field = w * ux ** a * uy ** b * uz ** c
            Mk = lattice_fft(field)[:, k[:, 0], k[:, 1], k[:, 2]]            # [model][nvox]
            coef = (1j ** n) * pw[0][:, a] * pw[1][:, b] * pw[2][:, c] / (
                math.factorial(a) * math.factorial(b) * math.factorial(c))
            if keep_n is not None:
                coef = np.where(keep_n[n], coef, 0.0)
            S += coef[None, :] * Mk
            if mode == DIFFUSE and n % 2 == 0:
                Sb += coef * np.mean(Mk, axis=0)
        F += phi[:, mu][None, :] * S
        Fb += phi[:, mu] * Sb
    if mode == DIFFUSE:
        F = F - np.where(bragg_vox, Fb, 0.0)[None, :]
    I = np.mean(np.abs(F) ** 2, axis=0) / model.natom
    return (I, F) if return_F else I


def truncation_bound(model, hkl, P, mode=DIFFUSE, F=None, chunk=4096):
    """Voxel-wise bound on |I_P - I| from the remainder |x|^(P+1)/(P+1)! of each atom's
    exp(i Q.u) (Section III C): dF = sum_j |w_j f_j| |Q.u_j|^(P+1)/(P+1)!; the Bragg term adds
    the supercell-mean of the same bound at integer H; then |I_P - I| <= (2|F| d + d^2)/N
    averaged over supercells, with F the exact (direct-sum) structure factor minus <F>.
    P is one order or one per Q point.  Evaluated in chunks of Q points to bound memory."""
    _, site = atom_list(model)
    nq = hkl.shape[0]
    Pq = np.broadcast_to(np.asarray(P, dtype=np.float64), (nq,))
    dFs = np.zeros((model.nmodels, nq))
    for s0 in range(0, nq, chunk):
        h = hkl[s0:s0 + chunk]
        Q = q_cart(h, model.lattice)
        qn = np.linalg.norm(Q, axis=1)
        f = np.stack([form_factor(int(model.ff_kind[s]), model.ff_coef[s], qn)
                      for s in range(model.nsite)], axis=1)
        ff = np.abs(f)[:, site]                             # [nq, natom]; b is in w
        for m in range(model.nmodels):
            u = model.disp[m].reshape(-1, 3).astype(np.float64)
            w = np.abs(displacive_weights(model, m))
            x = np.abs(Q @ u.T)                             # [nq, natom]
            Pc = Pq[s0:s0 + chunk][:, None]
            lf = np.array([math.lgamma(v + 2) for v in Pc[:, 0]])[:, None]
            rem = np.exp((Pc + 1) * np.log(np.maximum(x, 1e-300)) - lf)
            dFs[m, s0:s0 + chunk] = np.sum(ff * w[None, :] * rem, axis=1)
    if mode == DIFFUSE:
        dFs = dFs + is_integer_hkl(hkl)[None, :] * dFs.mean(axis=0)[None, :]
    if F is None:
        _, F = displacive_intensity_direct(model, hkl, mode, return_F=True)
    return np.mean(2 * np.abs(F) * dFs + dFs ** 2, axis=0) / model.natom
