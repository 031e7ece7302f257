"""CPU FP64 oracle for the gradient of chi^2 = sum_Q (I(Q) - I_target(Q))^2 (TOTAL mode).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

The paper defines no objective; the reading used here is unit weights and no scale factor.
The gradient is the chain rule of the direct sum (Eq. sf):
    dF_m(Q)/du_{j,alpha} = i Q_alpha w_j f_j exp(i Q . r_j)
    dI(Q)/du_{j,alpha}   = 2 / (M N) Re[ conj(F_m(Q)) dF_m(Q)/du_{j,alpha} ]
and for moments (Eqs. mag_sf, mag_intensity, mag_projection, |F_perp|^2 = F^H P F with
P = 1 - Q^ Q^T, or (2/3) 1 at Q = 0):
    dI(Q)/dM_{j,alpha}   = 2 C / (M N) Re[ conj((P F_m)_alpha) f_j exp(i Q . r_j) ]
"""
from __future__ import annotations

import numpy as np

from . import core


def _phases(model, hkl, u):
    frac, site = core.atom_list(model)
    Q = core.q_cart(hkl, model.lattice)
    t = hkl @ frac.T
    t = t - np.floor(t)
    ph = 2.0 * np.pi * t
    if u is not None:
        ph = ph + Q @ u.T
    f = core.site_form_factors(model, np.linalg.norm(Q, axis=1))[:, site]   # b f per atom
    return np.exp(1j * ph), f, Q


def displacive_chi2_grad(model, hkl, target, chunk=2048):
    """(chi2, grad [model][site][n1][n2][n3][3]) for displacive models in TOTAL mode."""
    I = core.displacive_intensity_direct(model, hkl, core.TOTAL)
    r = I - target
    chi2 = float(np.sum(r ** 2))
    MN = model.nmodels * model.natom
    grad = np.zeros((model.nmodels, model.natom, 3))
    for m in range(model.nmodels):
        u = model.disp[m].reshape(-1, 3).astype(np.float64)
        w = core.displacive_weights(model, m) / model.scat_len[core.atom_list(model)[1]]
        for s in range(0, hkl.shape[0], chunk):
            h = hkl[s:s + chunk]
            E, f, Q = _phases(model, h, u)
            a = E * (f * w[None, :])                                   # [nq, natom]
            F = a.sum(axis=1)
            # dchi2/du = sum_Q 2 r dI/du
            base = (2.0 * r[s:s + chunk])[:, None] * (2.0 / MN) * np.real(
                np.conj(F)[:, None] * 1j * a)                          # [nq, natom]
            grad[m] += base.T @ Q
    shape = (model.nmodels, model.nsite) + tuple(model.cells) + (3,)
    return chi2, grad.reshape(shape)


def magnetic_chi2_grad(model, hkl, target, chunk=2048):
    """(chi2, grad wrt moments [model][site][n1][n2][n3][3]) in TOTAL mode."""
    I = core.magnetic_intensity_direct(model, hkl, core.TOTAL)
    r = I - target
    chi2 = float(np.sum(r ** 2))
    MN = model.nmodels * model.natom
    grad = np.zeros((model.nmodels, model.natom, 3))
    for m in range(model.nmodels):
        M = model.spins[m].reshape(-1, 3).astype(np.float64)
        for s in range(0, hkl.shape[0], chunk):
            h = hkl[s:s + chunk]
            E, f, Q = _phases(model, h, None)
            a = E * f                                                  # [nq, natom]
            F = a @ M                                                  # [nq, 3]
            qn = np.linalg.norm(Q, axis=1)
            qhat = Q / np.where(qn > 0, qn, 1.0)[:, None]
            PF = F - qhat * np.sum(qhat * F, axis=1, keepdims=True)
            PF = np.where((qn > 0)[:, None], PF, (2.0 / 3.0) * F)
            coef = (2.0 * r[s:s + chunk]) * core.C_MAG * 2.0 / MN       # [nq]
            for al in range(3):
                grad[m][:, al] += np.real(np.conj(PF[:, al])[:, None] * a).T @ coef
    shape = (model.nmodels, model.nsite) + tuple(model.cells) + (3,)
    return chi2, grad.reshape(shape)
