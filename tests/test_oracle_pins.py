"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test names the passage it pins.  None of them re-types the oracle's own formula: each
compares against a different route to the same number (a double sum instead of a single sum,
a brute-force DFT instead of the FFT, a closed form, a symmetry, a finite difference).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import core, noise, adjoint
import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cart_positions(model, m=0, with_u=True):
    frac, site = core.atom_list(model)
    A = core.lattice_vectors(model.lattice)
    r = frac @ A
    if with_u and model.disp is not None:
        r = r + model.disp[m].reshape(-1, 3)
    return r, site


# ----------------------------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------------------------

def test_reciprocal_lattice_duality_and_hexagonal_d_spacing():
    """a_i . a*_j = 2 pi delta_ij (Section II definition of a*); hexagonal |Q| = 2 pi / d with
    the textbook 1/d^2 = 4 (h^2 + h k + k^2) / (3 a^2) + l^2 / c^2."""
    lat = (4.1, 4.6, 5.2, 84.0, 97.0, 101.0)
    A = core.lattice_vectors(lat)
    B = core.reciprocal_vectors(lat)
    assert np.allclose(A @ B.T, 2 * np.pi * np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.norm(A, axis=1), lat[:3])
    # Cartesian frame of the boundary: a along x, b in the xy plane, c with positive z
    assert abs(A[0, 1]) + abs(A[0, 2]) + abs(A[1, 2]) == 0.0 and A[0, 0] > 0 and A[2, 2] > 0
    cosg = np.dot(A[0], A[1]) / (lat[0] * lat[1])
    assert math.isclose(math.degrees(math.acos(cosg)), lat[5], rel_tol=1e-12)
    a, c = 3.3, 5.1
    hex_lat = (a, a, c, 90.0, 90.0, 120.0)
    for h, k, l in [(1, 0, 0), (1, 1, 0), (2, -1, 3), (0, 0, 2), (3, 2, 1)]:
        inv_d2 = 4.0 * (h * h + h * k + k * k) / (3 * a * a) + l * l / (c * c)
        q = np.linalg.norm(core.q_cart(np.array([[h, k, l]]), hex_lat))
        assert math.isclose(q, 2 * np.pi * math.sqrt(inv_d2), rel_tol=1e-12)


def test_form_factor_special_values():
    """s = 0 gives sum of amplitudes; large s leaves the constant term; <j0> of the magnetic
    workload at s^2 = 0.1 by hand."""
    g4 = np.array([1.0, 2.0, 3.0, 4.0, 10.0, 20.0, 30.0, 40.0, 0.5])
    assert math.isclose(core.form_factor(1, g4, np.array([0.0]))[0], 10.5)
    assert math.isclose(core.form_factor(1, g4, np.array([1e4]))[0], 0.5, abs_tol=1e-12)
    j0 = np.array(list(syn.J0_COEF) + [0, 0])
    q = 4 * np.pi * math.sqrt(0.1)
    want = 0.4 * math.exp(-1.5) + 0.6 * math.exp(-0.5) + 0.0 * math.exp(-0.1) + 0.0
    assert math.isclose(core.form_factor(2, j0, np.array([q]))[0], want, rel_tol=1e-14)


# ----------------------------------------------------------------------------------------------
# part 1: the direct sum
# ----------------------------------------------------------------------------------------------

def _double_sum_intensity(r, amp, site, ff_kind, ff_coef, lattice, hkl):
    """Eq. intensity_dble_sum: I = (1/N) sum_{j,k} a_j a_k exp(i Q.(r_j - r_k)), pure Python."""
    B = core.reciprocal_vectors(lattice)
    out = []
    for h in hkl:
        Q = h @ B
        qn = float(np.linalg.norm(Q))
        f = [core.form_factor(int(ff_kind[s]), ff_coef[s], np.array([qn]))[0] for s in site]
        acc = 0.0 + 0.0j
        for j in range(len(amp)):
            for k in range(len(amp)):
                acc += amp[j] * f[j] * amp[k] * f[k] * np.exp(1j * float(Q @ (r[j] - r[k])))
        out.append(acc.real / len(amp))
    return np.array(out)


def test_direct_sum_matches_double_sum():
    """Eq. intensity_sf with Eq. sf equals Eq. intensity_dble_sum (the factorisation of
    Section II), on <= 50 atoms with displacements, mixed form factors, triclinic cell."""
    m = syn.small_case(syn.DISP, cells=(3, 2, 2), nsite=4, nmodels=1, seed=5, sigma=0.2)
    frac, site = core.atom_list(m)
    r, _ = _cart_positions(m)
    w = core.displacive_weights(m, 0)
    rng = np.random.default_rng(0)
    hkl = rng.uniform(-2.5, 2.5, (12, 3))
    I1 = core.displacive_intensity_direct(m, hkl, core.TOTAL)
    I2 = _double_sum_intensity(r, w, site, m.ff_kind, m.ff_coef, m.lattice, hkl)
    assert frac.shape[0] <= 50
    np.testing.assert_allclose(I1, I2, rtol=1e-11, atol=1e-12 * np.max(I2))


def test_direct_sum_supercell_translation_invariance():
    """I(G) is unchanged when an atom moves by a supercell lattice vector, since
    exp(+-i G.n) = 1 (Section II); at an incommensurate Q it changes."""
    m = syn.small_case(syn.DISP, cells=(3, 4, 2), nsite=2, nmodels=1, seed=8)
    frac, site = core.atom_list(m)
    u = m.disp[0].reshape(-1, 3).astype(np.float64)
    w = core.displacive_weights(m, 0)
    G = np.array([[1, 2, -3], [4, -1, 0], [-2, 5, 3], [0, 0, 1]])
    hkl = G / np.array(m.cells)
    frac2 = frac.copy()
    frac2[5] += np.array(m.cells) * np.array([1, -2, 1])
    F1 = core.structure_factor(frac, u, w, site, m.ff_kind, m.ff_coef, m.lattice, hkl)
    F2 = core.structure_factor(frac2, u, w, site, m.ff_kind, m.ff_coef, m.lattice, hkl)
    np.testing.assert_allclose(F1, F2, rtol=1e-12, atol=1e-12)
    hq = np.array([[0.13, 0.41, -0.37]])
    Fa = core.structure_factor(frac, u, w, site, m.ff_kind, m.ff_coef, m.lattice, hq)
    Fb = core.structure_factor(frac2, u, w, site, m.ff_kind, m.ff_coef, m.lattice, hq)
    assert abs(Fa - Fb).max() > 1e-3


def test_undisplaced_fcc_closed_form():
    """Zero disorder, fcc with f = 1: I(H) = N for unmixed hkl, 0 for mixed hkl, and
    I(G) = 0 off the unit-cell Bragg positions (k != 0), for the direct sum and both FFT
    routes (occupancy with delta = 1, displacive with u = 0)."""
    cells = (4, 3, 2)
    m = syn.displacive_fcc(cells=cells, sigma=0.0, seed=1)
    m.disp[:] = 0.0
    G = np.stack(np.meshgrid(np.arange(-8, 8), np.arange(-6, 6), np.arange(-4, 4),
                             indexing="ij"), -1).reshape(-1, 3)
    hkl = G / np.array(cells)
    integer = np.all(np.mod(G, cells) == 0, axis=1)
    H = (G // np.array(cells))
    unmixed = np.all(np.mod(H, 2) == 0, axis=1) | np.all(np.mod(H, 2) == 1, axis=1)
    want = np.where(integer & unmixed, m.natom, 0.0)
    I_dir = core.displacive_intensity_direct(m, hkl, core.TOTAL)
    np.testing.assert_allclose(I_dir, want, atol=1e-9 * m.natom)
    I_fft = core.displacive_intensity_fft(m, G, core.TOTAL, P=3)
    np.testing.assert_allclose(I_fft, want, atol=1e-9 * m.natom)
    m.occ = np.ones((1, 4) + cells, dtype=np.uint8)
    I_occ = core.occupancy_intensity_fft(m, G, core.TOTAL)
    np.testing.assert_allclose(I_occ, want, atol=1e-9 * m.natom)
    # DIFFUSE with delta = 1 and u = 0 has nothing left
    assert np.max(np.abs(core.occupancy_intensity_fft(m, G, core.DIFFUSE))) < 1e-9
    assert np.max(np.abs(core.occupancy_intensity_direct(m, hkl, core.DIFFUSE))) < 1e-9 * m.natom


@pytest.mark.parametrize("kind", [syn.OCC, syn.SPIN, syn.DISP])
def test_friedel_symmetry(kind):
    """I(Q) = I(-Q) for real amplitudes (all three disorder types, both modes)."""
    m = syn.small_case(kind, cells=(3, 4, 3), nsite=3, nmodels=2, seed=21)
    rng = np.random.default_rng(3)
    hkl = rng.uniform(-2, 2, (20, 3))
    hkl[:4] = np.rint(hkl[:4])                 # include integer (Bragg) points
    both = np.concatenate([hkl, -hkl])
    for mode in (core.TOTAL, core.DIFFUSE):
        if kind == syn.OCC:
            I = core.occupancy_intensity_direct(m, both, mode)
        elif kind == syn.SPIN:
            I = core.magnetic_intensity_direct(m, both, mode)
        else:
            I = core.displacive_intensity_direct(m, both, mode)
        np.testing.assert_allclose(I[:20], I[20:], rtol=1e-10, atol=1e-12 * I.max())


def test_magnetic_projection_special_cases():
    """Eqs. mag_intensity, mag_projection: a single moment parallel to Q^ scatters nothing; a
    moment perpendicular to Q^ gives C |F|^2 / N; at Q = 0 the orientational average 2/3."""
    m = syn.small_case(syn.SPIN, cells=(1, 1, 1), nsite=1, nmodels=1, seed=2)
    m.ff_kind[:] = 0
    m.scat_len[:] = 1.0
    hkl = np.array([[0.3, -0.2, 0.7]])
    Q = core.q_cart(hkl, m.lattice)[0]
    qhat = Q / np.linalg.norm(Q)
    perp = np.cross(qhat, [0.3, 0.5, 0.1])
    perp /= np.linalg.norm(perp)
    m.spins = np.zeros((1, 1, 1, 1, 1, 3), dtype=np.float32)
    m.spins[..., :] = qhat.astype(np.float32)
    assert core.magnetic_intensity_direct(m, hkl)[0] < 1e-12
    m.spins[..., :] = perp.astype(np.float32)
    s = float(np.linalg.norm(m.spins[0, 0, 0, 0, 0].astype(np.float64)))
    assert math.isclose(core.magnetic_intensity_direct(m, hkl)[0], core.C_MAG * s * s, rel_tol=1e-9)
    I0 = core.magnetic_intensity_direct(m, np.zeros((1, 3)))[0]
    assert math.isclose(I0, core.C_MAG * (2.0 / 3.0) * s * s, rel_tol=1e-9)
    assert core.C_MAG == 0.07265


# ----------------------------------------------------------------------------------------------
# part 2: the FFT method
# ----------------------------------------------------------------------------------------------

def test_lattice_fft_matches_brute_force_dft():
    """Eq. fft (sign +i, no normalisation) against an O(n^6) loop, on a 4 x 3 x 5 grid; delta,
    constant and plane-wave special cases."""
    rng = np.random.default_rng(1)
    n = (4, 3, 5)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = core.lattice_fft(x)
    for k in itertools.product(*(range(a) for a in n)):
        acc = 0.0 + 0.0j
        for R in itertools.product(*(range(a) for a in n)):
            acc += x[R] * np.exp(2j * np.pi * sum(k[a] * R[a] / n[a] for a in range(3)))
        assert abs(X[k] - acc) < 1e-11
    d = np.zeros(n)
    d[1, 2, 3] = 1.0
    kk = np.stack(np.meshgrid(*(np.arange(a) for a in n), indexing="ij"), -1)
    want = np.exp(2j * np.pi * (kk[..., 0] * 1 / 4 + kk[..., 1] * 2 / 3 + kk[..., 2] * 3 / 5))
    np.testing.assert_allclose(core.lattice_fft(d), want, atol=1e-12)
    c = core.lattice_fft(np.ones(n))
    assert abs(c[0, 0, 0] - 60) < 1e-12 and np.abs(c).sum() - 60 < 1e-10
    R = np.stack(np.meshgrid(*(np.arange(a) for a in n), indexing="ij"), -1)
    k0 = (1, 2, 4)
    pw = np.exp(-2j * np.pi * sum(k0[a] * R[..., a] / n[a] for a in range(3)))
    P = core.lattice_fft(pw)
    assert abs(P[k0] - 60) < 1e-10 and np.abs(P).sum() - 60 < 1e-9


@pytest.mark.parametrize("shape", [(7, 20, 32), (32, 7, 20), (20, 32, 7)])
def test_lattice_fft_at_the_kernel_sizes_matches_separable_dft(shape):
    """Eq. fft at the sizes the GPU transforms specialise (radix 7, 20 = 4 * 5, 32 = 4 * 4 * 2),
    each size on each axis: the oracle's transform equals the definition evaluated one axis at
    a time, X = sum_R x_R prod_a exp(2 pi i k_a R_a / n_a), with the phase of each 1-D matrix
    reduced exactly (k R mod n in integers) before the exponential."""
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    mats = []
    for n in shape:
        kR = np.mod(np.outer(np.arange(n), np.arange(n)), n)
        mats.append(np.exp(2j * np.pi * kR / n))
    want = np.einsum("ai,bj,ck,ijk->abc", mats[0], mats[1], mats[2], x)
    got = core.lattice_fft(x)
    assert np.max(np.abs(got - want)) < 1e-10 * np.max(np.abs(want))
    # a plane wave exp(-2 pi i k0.R/n) lands in the single bin k0 with weight n1 n2 n3
    k0 = tuple(n - 2 for n in shape)
    R = np.stack(np.meshgrid(*(np.arange(n) for n in shape), indexing="ij"), -1)
    pw = np.exp(-2j * np.pi * sum(k0[a] * R[..., a] / shape[a] for a in range(3)))
    P = core.lattice_fft(pw)
    N = float(np.prod(shape))
    assert abs(P[k0] - N) < 1e-9 * N and np.abs(P).sum() - N < 1e-8 * N


def test_parseval():
    """sum_k |X_k|^2 = n1 n2 n3 sum_R |x_R|^2 for every transformed field."""
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 6, 5, 4))
    X = core.lattice_fft(x)
    np.testing.assert_allclose(np.sum(np.abs(X) ** 2, axis=(1, 2, 3)),
                               120 * np.sum(x ** 2, axis=(1, 2, 3)), rtol=1e-12)


def _grid_G(model):
    return model.qgrid.g_index(model.cells)


@pytest.mark.parametrize("mode", [0, 1])
def test_fft_method_equals_direct_sum_occupancy(mode):
    """'Calculations using the DFT and the FFT gave identical results' (Section IV) for
    compositional disorder, Eqs. comp_sf_diffuse..comp_diffuse_intensity: equal to rounding."""
    m = syn.small_case(syn.OCC, cells=(4, 3, 5), nsite=3, nmodels=2, seed=31)
    G = _grid_G(m)
    hkl = G / np.array(m.cells)
    I_fft = core.occupancy_intensity_fft(m, G, mode)
    I_dir = core.occupancy_intensity_direct(m, hkl, mode)
    np.testing.assert_allclose(I_fft, I_dir, rtol=1e-9, atol=1e-11 * I_dir.max())


@pytest.mark.parametrize("mode", [0, 1])
def test_fft_method_equals_direct_sum_magnetic(mode):
    """Same for magnetic disorder, Eqs. mag_sf..mag_projection, incl. the G = 0 voxel."""
    m = syn.small_case(syn.SPIN, cells=(3, 4, 3), nsite=3, nmodels=2, seed=32)
    G = _grid_G(m)
    assert np.any(np.all(G == 0, axis=1))
    hkl = G / np.array(m.cells)
    I_fft = core.magnetic_intensity_fft(m, G, mode)
    I_dir = core.magnetic_intensity_direct(m, hkl, mode)
    np.testing.assert_allclose(I_fft, I_dir, rtol=1e-9, atol=1e-11 * I_dir.max())


@pytest.mark.parametrize("mode,P", [(0, 4), (1, 4), (1, 8), (0, 14)])
def test_taylor_fft_within_remainder_bound(mode, P):
    """Section III C: the order-P Taylor FFT method differs from the exact direct sum by no
    more than the remainder bound, voxel by voxel; at high order it converges to rounding."""
    m = syn.small_case(syn.DISP, cells=(3, 4, 2), nsite=3, nmodels=2, seed=33, sigma=0.15)
    G = _grid_G(m)
    hkl = G / np.array(m.cells)
    I_dir, F = core.displacive_intensity_direct(m, hkl, mode, return_F=True)
    I_fft = core.displacive_intensity_fft(m, G, mode, P=P)
    bound = core.truncation_bound(m, hkl, P, mode, F=F)
    assert np.all(np.abs(I_fft - I_dir) <= bound * (1 + 1e-9) + 1e-12 * I_dir.max())
    if P >= 14:
        assert np.max(np.abs(I_fft - I_dir)) < 1e-9 * I_dir.max()
    else:
        assert np.max(np.abs(I_fft - I_dir)) > 1e-14   # the truncation is visible


def test_monomial_enumeration_counts():
    """(n+1)(n+2)/2 FFTs for order n; the fifth-order pure-displacive example needs 55 FFTs
    (Section IV: the order-0 field of a pure displacive model is constant)."""
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        gold = json.load(f)
    mons = core.monomials(5)
    assert len(mons) - 1 == gold["ffts_fifth_order_displacive"]["value"] == 55
    for P in range(12):
        mons = core.monomials(P)
        assert len(set(mons)) == len(mons) == (P + 1) * (P + 2) * (P + 3) // 6
        for n in range(P + 1):
            assert sum(1 for t in mons if sum(t) == n) == (n + 1) * (n + 2) // 2
        assert [sum(t) for t in mons] == sorted(sum(t) for t in mons)


def test_taylor_order_and_x_max():
    """The chosen order is the first whose remainder bound x^(P+1)/(P+1)! is below eps, and
    x_max (box corners) equals the brute-force maximum of |Q.u| over every grid point."""
    for x, eps in [(4.6, 1e-8), (9.7, 1e-5), (0.3, 1e-12), (1.0, 0.3)]:
        P = core.taylor_order(x, eps)
        assert x ** (P + 1) / math.factorial(P + 1) <= eps
        if P > 0:
            assert x ** P / math.factorial(P) > eps
    m = syn.small_case(syn.DISP, cells=(3, 2, 2), nsite=2, nmodels=2, seed=4, sigma=0.2)
    Q = core.q_cart(m.qgrid.hkl(), m.lattice)
    u = m.disp.reshape(-1, 3).astype(np.float64)
    assert math.isclose(core.x_max(m, m.qgrid), float(np.max(np.abs(Q @ u.T))), rel_tol=1e-12)


def test_zone_taylor_orders_bound_every_voxel():
    """Per-zone reading of the remainder bound (Section III C): at every voxel the zone's order
    keeps the largest per-atom remainder |Q.u_j|^(P+1)/(P+1)! (brute force over all atoms) below
    eps; no zone exceeds the grid order, the zone of largest |Q| takes it when the bound
    |Q||u| is tight enough, and the zones near Q = 0 take a lower one."""
    m = syn.small_case(syn.DISP, cells=(3, 4, 2), nsite=3, nmodels=2, seed=33, sigma=0.15)
    eps = 1e-6
    pv, P = core.zone_taylor_orders(m, m.qgrid, eps)
    Q = core.q_cart(m.qgrid.hkl(), m.lattice)
    u = m.disp.reshape(-1, 3).astype(np.float64)
    x = np.max(np.abs(Q @ u.T), axis=1)                      # per voxel, all atoms
    lf = np.array([math.lgamma(p + 2) for p in pv])
    assert np.all((pv + 1) * np.log(np.maximum(x, 1e-300)) - lf <= math.log(eps) + 1e-12)
    assert pv.max() <= P and pv.min() < P
    qn = np.linalg.norm(Q, axis=1)
    assert pv[np.argmin(qn)] < pv[np.argmax(qn)]


@pytest.mark.parametrize("mode", [0, 1])
def test_zone_orders_equal_fixed_order_per_voxel(mode):
    """Masking by zone order: each voxel of the per-zone result equals the fixed-order method
    run at that voxel's own order (a separate run per order, Bragg term included), and stays
    within the per-voxel remainder bound of the exact direct sum."""
    m = syn.small_case(syn.DISP, cells=(3, 4, 2), nsite=3, nmodels=2, seed=34, sigma=0.15)
    pv, P = core.zone_taylor_orders(m, m.qgrid, 1e-5)
    G = _grid_G(m)
    I_z = core.displacive_intensity_fft(m, G, mode, P=P, P_vox=pv)
    assert len(np.unique(pv)) >= 2
    for p in np.unique(pv):
        sel = pv == p
        I_p = core.displacive_intensity_fft(m, G[sel], mode, P=int(p))
        assert np.allclose(I_z[sel], I_p, rtol=1e-12, atol=1e-13 * np.abs(I_z).max())
    hkl = G / np.array(m.cells)
    I_dir, F = core.displacive_intensity_direct(m, hkl, mode, return_F=True)
    bound = core.truncation_bound(m, hkl, pv, mode, F=F)
    assert np.all(np.abs(I_z - I_dir) <= bound * (1 + 1e-9) + 1e-12 * I_dir.max())


def test_gaussian_displacements_laue_closed_form():
    """Independent Gaussian displacements (sigma per Cartesian component), f = 1: at every
    k != 0 voxel E[I] = 1 - exp(-Q^2 sigma^2); at allowed unit-cell Bragg positions the total
    intensity is N exp(-Q^2 sigma^2) + 1 - exp(-Q^2 sigma^2).  Checked on the 8^3 fcc
    workload over the full 64^3 grid (speckle averages out over the volume)."""
    m = syn.displacive_fcc(cells=(8, 8, 8), sigma=0.1, seed=1)
    G = _grid_G(m)
    hkl = G / 8.0
    I = core.displacive_intensity_direct(m, hkl, core.TOTAL)
    Q2 = np.sum(core.q_cart(hkl, m.lattice) ** 2, axis=1)
    laue = 1.0 - np.exp(-Q2 * 0.01)
    off = ~np.all(np.mod(G, 8) == 0, axis=1)
    ratio = np.mean(I[off] / laue[off])
    assert abs(ratio - 1.0) < 5.0 / math.sqrt(off.sum() / 2)
    H = G // 8
    onb = (~off) & (np.all(H % 2 == 0, axis=1) | np.all(H % 2 == 1, axis=1))
    low = onb & (Q2 * 0.01 < 0.5)
    want = m.natom * np.exp(-Q2[low] * 0.01) + laue[low]
    np.testing.assert_allclose(I[low], want, rtol=0.15)


# ----------------------------------------------------------------------------------------------
# noise reduction
# ----------------------------------------------------------------------------------------------

def test_lanczos_weights_and_normalisation():
    """Eqs. weight_sinc, windowed_sinc, lanczos: for m = 2 at commensurate Q the 1D taps are
    1 (centre) and (2/pi)^2 (neighbours), the normalised centre 1/(1 + 8/pi^2); the 3D weight
    is the product of 1D ones; constant I(G) is reproduced exactly; the 1/m' variant with
    m = 2 is the squared sinc (Fejer) kernel."""
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        gold = json.load(f)
    d = np.array([[0.0, 0, 0], [1, 0, 0], [2, 0, 0], [1, 1, 0], [1, -1, 1]])
    W = noise.lanczos_weight(d, 2) / noise.lanczos_weight(np.zeros((1, 3)), 2)[0]
    nb = gold["lanczos_m2_neighbour_weight"]["value"]
    assert math.isclose(nb, (2 / math.pi) ** 2, rel_tol=1e-5)
    np.testing.assert_allclose(W, [1, nb, 0, nb ** 2, nb ** 3], rtol=1e-5, atol=1e-15)
    w1 = np.array([nb, 1.0, nb])
    assert math.isclose(1.0 / w1.sum(), gold["lanczos_m2_centre_normalised"]["value"], rel_tol=1e-4)
    Q = np.array([[3.0, -2.0, 5.0], [0.25, 1.75, -3.5], [7.3, 0.1, -0.9]])
    out = noise.lanczos_resample(lambda G: np.full(G.shape[0], 4.25), Q, 3)
    np.testing.assert_allclose(out, 4.25, rtol=1e-13)
    dd = np.arange(-7, 8, dtype=np.float64)
    w8 = noise.lanczos_weight(np.stack([dd, 0 * dd, 0 * dd], -1), 2, 8)
    fej = noise.sinc(np.pi * dd / 8) ** 2
    np.testing.assert_allclose(w8 / w8[7], fej, rtol=1e-12, atol=1e-15)


def test_sphere_cutoff_is_the_fourier_transform_of_a_ball():
    """Section V B, spherical cutoff: sin x/x^3 - cos x/x^2 (x = q r_c) is the Fourier transform of
    the ball |r| < r_c divided by 4 pi r_c^3 -- checked against a radial quadrature of
    int_0^rc 4 pi r^2 sin(q r)/(q r) dr, and its x -> 0 limit 1/3 (the ball volume)."""
    from scipy.integrate import quad
    rc = 7.3
    for q in (1e-6, 0.05, 0.4, 1.3, 2.9):
        ball = quad(lambda r: 4 * math.pi * r * r * (math.sin(q * r) / (q * r)), 0.0, rc, limit=200)[0]
        assert math.isclose(float(noise.sphere_weight(np.array([q]), rc)[0]) * 4 * math.pi * rc ** 3, ball,
                            rel_tol=1e-9, abs_tol=1e-9 * rc ** 3)
    assert math.isclose(float(noise.sphere_weight(np.array([0.0]), rc)[0]), 1.0 / 3.0)


def test_sphere_resample_constant_and_isotropy():
    """The spherical window reproduces a constant intensity, depends only on |Q - G| (cubic cell:
    permuting the axes of I(G) and of Q permutes nothing in the result), and the inscribed radius
    of a cubic supercell is half its edge."""
    m = syn.small_case(syn.OCC, cells=(4, 4, 4), nsite=1, nmodels=1, seed=3)
    m.lattice = (5.0, 5.0, 5.0, 90.0, 90.0, 90.0)
    assert math.isclose(noise.inscribed_radius(m), 10.0, rel_tol=1e-12)
    rng = np.random.default_rng(4)
    Q = rng.uniform(-6, 6, (40, 3))
    out = noise.sphere_resample(m, lambda G: np.full(G.shape[0], 2.5), Q, 2)
    assert np.allclose(out, 2.5, rtol=1e-12)
    f = lambda G: np.cos(0.3 * G[:, 0]) + 0.1 * G[:, 1] ** 2 + np.sin(G[:, 2])
    fp = lambda G: f(G[:, [1, 2, 0]])
    a = noise.sphere_resample(m, f, Q, 2)
    b = noise.sphere_resample(m, fp, Q[:, [2, 0, 1]], 2)
    assert np.allclose(a, b, rtol=1e-12)


def test_lanczos_resample_separable():
    """Separable application along each axis in turn (Section V B) equals the 3D sum."""
    rng = np.random.default_rng(7)
    table = {}

    def I_at(G):
        out = np.empty(G.shape[0])
        for i, g in enumerate(map(tuple, G)):
            if g not in table:
                table[g] = rng.random()
            out[i] = table[g]
        return out

    Q = np.array([[2.0, -1.0, 0.0], [4.0, 4.0, -3.0]])
    full = noise.lanczos_resample(I_at, Q, 2)
    for qi, q in enumerate(Q):
        taps = np.arange(-1, 2)
        w = noise.lanczos_weight(np.stack([taps, 0 * taps, 0 * taps], -1).astype(float), 2)
        w = w / w.sum()
        acc = 0.0
        for a, wa in zip(taps, w):
            for b, wb in zip(taps, w):
                for c, wc in zip(taps, w):
                    acc += wa * wb * wc * I_at(np.array([[q[0] + a, q[1] + b, q[2] + c]]).astype(int))[0]
        assert math.isclose(full[qi], acc, rel_tol=1e-12)


@pytest.mark.parametrize("disorder", ["occ", "spin"])
def test_subbox_single_cell_closed_form(disorder):
    """n_sb = 1: every box is one unit cell, so I = (1/(ncell nsite)) sum_R |sum_mu phi_mu x_R|^2
    (cell-incoherent sum; Section V A with the smallest box)."""
    kind = syn.OCC if disorder == "occ" else syn.SPIN
    m = syn.small_case(kind, cells=(3, 2, 3), nsite=3, nmodels=2, seed=41)
    rng = np.random.default_rng(5)
    hkl = rng.uniform(-1.5, 1.5, (7, 3))
    I = noise.subbox_intensity(m, disorder, core.DIFFUSE, 1, hkl)
    x = noise.subbox_fields(m, disorder, core.DIFFUSE)              # [model][site][...][c]
    Q = core.q_cart(hkl, m.lattice)
    f = core.site_form_factors(m, np.linalg.norm(Q, axis=1)) / m.scat_len[None, :]
    t = hkl @ m.sites.T
    phi = f * np.exp(2j * np.pi * t)                                # [nq, nsite]
    acc = np.zeros(hkl.shape[0])
    for mm in range(m.nmodels):
        xr = x[mm].reshape(m.nsite, -1, x.shape[-1])                # [site][R][c]
        F = np.einsum("qs,src->qrc", phi, xr)                        # per cell
        if disorder == "spin":
            for r in range(F.shape[1]):
                acc += core.perp_sq(F[:, r, :], Q)
        else:
            acc += np.sum(np.abs(F[..., 0]) ** 2, axis=1)
    want = acc / (m.nmodels * m.ncell * m.nsite)
    if disorder == "spin":
        want = core.C_MAG * want
    np.testing.assert_allclose(I, want, rtol=1e-10)


def test_subbox_pair_sum_form():
    """The triangular-cutoff reading of Section V A: sum over origins of |F_o|^2 equals
    sum_{mu,nu} phi_mu conj(phi_nu) sum_Delta w(Delta) exp(iQ.(Delta + r_mu - r_nu)) C(Delta),
    w(Delta) = prod_alpha (n_sb - |Delta_alpha|), C(Delta) = sum_R x_{R+Delta,mu} x_{R,nu}
    (periodic), at arbitrary (incommensurate) Q."""
    m = syn.small_case(syn.OCC, cells=(5, 4, 6), nsite=2, nmodels=1, seed=42)
    nsb = 2
    rng = np.random.default_rng(9)
    hkl = rng.uniform(-1.2, 1.2, (5, 3))
    I = noise.subbox_intensity(m, "occ", core.TOTAL, nsb, hkl)
    x = noise.subbox_fields(m, "occ", core.TOTAL)[0, ..., 0]        # [site][n1][n2][n3]
    Q = core.q_cart(hkl, m.lattice)
    f = core.site_form_factors(m, np.linalg.norm(Q, axis=1)) / m.scat_len[None, :]
    acc = np.zeros(hkl.shape[0], dtype=complex)
    rng_d = range(-nsb + 1, nsb)
    for mu in range(m.nsite):
        for nu in range(m.nsite):
            for D in itertools.product(rng_d, rng_d, rng_d):
                w = np.prod([nsb - abs(d) for d in D])
                C = np.sum(np.roll(x[mu], shift=[-d for d in D], axis=(0, 1, 2)) * x[nu])
                ph = np.exp(2j * np.pi * (hkl @ (np.array(D) + m.sites[mu] - m.sites[nu])))
                acc += f[:, mu] * f[:, nu] * w * C * ph
    want = acc.real / (m.ncell * m.nsite * nsb ** 3)
    np.testing.assert_allclose(I, want, rtol=1e-10)


def _box_sf_closed_form(m, hkl, nsb):
    """sum_{d in [0, nsb)^3} exp(2 pi i hkl.d), a product of three geometric series."""
    out = np.ones(hkl.shape[0], dtype=complex)
    for a in range(3):
        z = np.exp(2j * np.pi * hkl[:, a])
        near = np.abs(z - 1.0) < 1e-12
        safe = np.where(near, 0.5, z)
        out *= np.where(near, nsb, (1.0 - safe ** nsb) / (1.0 - safe))
    return out


def test_subbox_displacive_without_displacements_is_occupational():
    """u = 0: the displacive sub-box (amplitude b delta exp(i Q.u), DIFFUSE minus b <delta>)
    reduces to the occupational one (b delta, DIFFUSE b (delta - c)) at any Q and origin set."""
    m = syn.small_case(syn.DISP, cells=(4, 3, 5), nsite=3, nmodels=2, seed=61)
    m.disp = np.zeros_like(m.disp)
    rng = np.random.default_rng(3)
    hkl = rng.uniform(-1.7, 1.7, (6, 3))
    org = syn.random_origins(rng, m.nmodels, m.cells, 5)
    for mode in (core.TOTAL, core.DIFFUSE):
        for origins in (None, org):
            a = noise.subbox_intensity(m, "disp", mode, 2, hkl, origins)
            b = noise.subbox_intensity(m, "occ", mode, 2, hkl, origins)
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14)


def test_subbox_displacive_rigid_shift_ensemble():
    """Supercell 0 shifted rigidly by u0, supercell 1 by -u0 (no occupancies): |F_o| does not
    change (TOTAL equals the undisplaced result), T_mu(Q) = cos(Q.u0) on every site, so each
    atom scatters i b sin(Q.u0) exp(i Q.r) and DIFFUSE = sin^2(Q.u0) TOTAL(u = 0); the box sum
    of one cell-uniform box is the closed-form geometric series."""
    m = syn.small_case(syn.DISP, cells=(3, 4, 3), nsite=1, nmodels=2, seed=62)
    m.ff_kind = np.zeros(1, dtype=np.int32)
    u0 = np.array([0.11, -0.07, 0.05])
    m.disp = np.zeros_like(m.disp)
    m.disp[0] = u0
    m.disp[1] = -u0
    rng = np.random.default_rng(4)
    hkl = rng.uniform(-2.0, 2.0, (8, 3))
    nsb = 2
    tot = noise.subbox_intensity(m, "disp", core.TOTAL, nsb, hkl)
    dif = noise.subbox_intensity(m, "disp", core.DIFFUSE, nsb, hkl)
    # one site, constant form factor: |F_o| = b |box series|, the same for every origin
    want0 = m.scat_len[0] ** 2 * np.abs(_box_sf_closed_form(m, hkl, nsb)) ** 2 / nsb ** 3
    np.testing.assert_allclose(tot, want0, rtol=1e-12)
    qu = core.q_cart(hkl, m.lattice) @ m.disp[0, 0, 0, 0, 0].astype(np.float64)
    np.testing.assert_allclose(dif, np.sin(qu) ** 2 * want0, rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("mode", [0, 1])
def test_subbox_whole_supercell_box_is_the_direct_sum(mode):
    """n_sb = n: one box covers the whole supercell, so at a supercell Bragg position (where
    exp(i G.R) is periodic) every origin gives F of the direct sum of its supercell (two origins
    per supercell here, so that the supercells weigh equally), and DIFFUSE gives F - <F> with
    <F> of Eq. bragg_sf_disp: I equals core.displacive_intensity_direct."""
    m = syn.small_case(syn.DISP, cells=(3, 3, 3), nsite=2, nmodels=2, seed=63, sigma=0.12)
    rng = np.random.default_rng(6)
    G = rng.integers(-5, 6, (6, 3))
    G[0] = (3, 0, -3)                      # an integer hkl: the Bragg term is nonzero there
    hkl = G / 3.0
    org = np.array([[0, 1, 2, 0], [1, 0, 0, 0], [1, 2, 2, 1], [0, 0, 0, 0]], dtype=np.int32)
    got = noise.subbox_intensity(m, "disp", mode, 3, hkl, org)
    want = core.displacive_intensity_direct(m, hkl, mode)
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-12 * want.max())


def test_subbox_origin_sets_average_linearly():
    """The random-origin estimate is the mean of one-origin estimates, and the list of every
    lattice point of every supercell gives the every-lattice-point variant."""
    m = syn.small_case(syn.SPIN, cells=(3, 2, 4), nsite=2, nmodels=2, seed=64)
    rng = np.random.default_rng(7)
    hkl = rng.uniform(-1.0, 1.0, (4, 3))
    org = syn.random_origins(rng, m.nmodels, m.cells, 4)
    many = noise.subbox_intensity(m, "spin", core.DIFFUSE, 2, hkl, org)
    ones = [noise.subbox_intensity(m, "spin", core.DIFFUSE, 2, hkl, org[i:i + 1]) for i in range(4)]
    np.testing.assert_allclose(many, np.mean(ones, axis=0), rtol=1e-12)
    np.testing.assert_allclose(noise.subbox_intensity(m, "spin", core.TOTAL, 2, hkl, noise.all_origins(m)),
                               noise.subbox_intensity(m, "spin", core.TOTAL, 2, hkl), rtol=1e-12)
    cov = syn.covering_origins(rng, m.nmodels, m.cells, 2)
    for mm in range(m.nmodels):
        hit = np.zeros(m.cells, dtype=bool)
        for row in cov[cov[:, 0] == mm]:
            idx = [np.mod(row[1 + a] + np.arange(2), m.cells[a]) for a in range(3)]
            hit[np.ix_(*idx)] = True
        assert hit.all()


# ----------------------------------------------------------------------------------------------
# Debye-Waller factor and the magnetic + displacive coupling (Eqs. dw, mag_sf)
# ----------------------------------------------------------------------------------------------

def test_debye_waller_closed_forms():
    """T_mu(Q): 1 without displacements; cos(Q.u0) for a site shifted rigidly by u0 (the even
    part of exp(i Q.u0)); exp(-sigma^2 |Q|^2 / 2) for isotropic Gaussian displacements, within
    the sampling error of 2 x 12^3 atoms per site; |T| <= 1."""
    m = syn.pyrochlore_mag_disp(cells=(12, 12, 12), sigma=0.06, nsite=3, nmodels=2, seed=65)
    rng = np.random.default_rng(8)
    hkl = rng.uniform(-5.0, 5.0, (40, 3))
    Q = core.q_cart(hkl, m.lattice)
    T = core.debye_waller(m, hkl)
    assert np.all(np.abs(T) <= 1.0 + 1e-12)
    gauss = np.exp(-0.5 * 0.06 ** 2 * np.sum(Q * Q, axis=1))
    nsample = m.nmodels * m.ncell
    assert np.max(np.abs(T - gauss[:, None])) < 5.0 * math.sqrt(0.5 / nsample)
    u0 = np.array([[0.2, -0.1, 0.05], [0.0, 0.3, 0.0], [-0.15, 0.0, 0.25]])
    m.disp = np.broadcast_to(u0[None, :, None, None, None, :], m.disp.shape).astype(np.float32)
    np.testing.assert_allclose(core.debye_waller(m, hkl), np.cos(Q @ m.disp[0, :, 0, 0, 0].astype(np.float64).T),
                               rtol=1e-12, atol=1e-14)
    m.disp = np.zeros_like(m.disp)
    np.testing.assert_array_equal(core.debye_waller(m, hkl), 1.0)


def test_magnetic_debye_waller_coupling():
    """Eq. mag_sf with T_mu: without displacements T = 1 and the result is the uncoupled one;
    with one site shifted rigidly by u0 the intensity is cos^2(Q.u0) times the uncoupled one
    at any Q; and the FFT method with T_mu per voxel equals the direct sum at the Bragg
    positions of the supercell (TOTAL and DIFFUSE)."""
    m = syn.pyrochlore_mag_disp(cells=(3, 4, 3), sigma=0.08, nsite=1, nmodels=2, seed=66)
    rng = np.random.default_rng(9)
    hkl = rng.uniform(-2.0, 2.0, (9, 3))
    base = core.magnetic_intensity_direct(m, hkl, core.TOTAL)
    u0 = np.array([0.13, 0.04, -0.09])
    keep = m.disp
    m.disp = np.zeros_like(keep)
    np.testing.assert_allclose(core.magnetic_intensity_direct(m, hkl, core.TOTAL, dw=True), base, rtol=1e-13)
    m.disp[:] = u0
    qu = core.q_cart(hkl, m.lattice) @ m.disp[0, 0, 0, 0, 0].astype(np.float64)
    np.testing.assert_allclose(core.magnetic_intensity_direct(m, hkl, core.TOTAL, dw=True),
                               np.cos(qu) ** 2 * base, rtol=1e-12)
    m3 = syn.pyrochlore_mag_disp(cells=(3, 4, 3), sigma=0.08, nsite=3, nmodels=2, seed=66)
    G = rng.integers(-7, 8, (30, 3))
    G[0] = (3, -4, 6)
    hk = G / np.asarray(m3.cells, dtype=float)
    for mode in (core.TOTAL, core.DIFFUSE):
        d = core.magnetic_intensity_direct(m3, hk, mode, dw=True)
        f = core.magnetic_intensity_fft(m3, G, mode, dw=True)
        np.testing.assert_allclose(f, d, rtol=1e-10, atol=1e-12 * d.max())
        assert not np.allclose(d, core.magnetic_intensity_direct(m3, hk, mode), rtol=1e-3)


# ----------------------------------------------------------------------------------------------
# gradient
# ----------------------------------------------------------------------------------------------

def _fd(fun, model, arr_name, index, h=1e-5):
    arr = getattr(model, arr_name)
    base = arr.astype(np.float64)
    plus, minus = base.copy(), base.copy()
    plus[index] += h
    minus[index] -= h
    setattr(model, arr_name, plus)
    fp = fun()
    setattr(model, arr_name, minus)
    fm = fun()
    setattr(model, arr_name, arr)
    return (fp - fm) / (2 * h)


def test_displacive_gradient_finite_differences():
    """Analytic chi^2 gradient vs central differences (FP64, h = 1e-5 A)."""
    m = syn.small_case(syn.DISP, cells=(2, 3, 2), nsite=2, nmodels=2, seed=51, sigma=0.1)
    t = syn.small_case(syn.DISP, cells=(2, 3, 2), nsite=2, nmodels=2, seed=52, sigma=0.07)
    hkl = np.random.default_rng(1).uniform(-2, 2, (40, 3))
    target = core.displacive_intensity_direct(t, hkl, core.TOTAL)
    chi2, grad = adjoint.displacive_chi2_grad(m, hkl, target)
    fun = lambda: float(np.sum((core.displacive_intensity_direct(m, hkl, core.TOTAL) - target) ** 2))
    assert math.isclose(chi2, fun(), rel_tol=1e-12)
    for idx in [(0, 0, 0, 0, 0, 0), (1, 1, 1, 2, 1, 2), (0, 1, 1, 0, 0, 1), (1, 0, 0, 1, 1, 0)]:
        fd = _fd(fun, m, "disp", idx)
        assert math.isclose(grad[idx], fd, rel_tol=2e-5, abs_tol=1e-7 * np.abs(grad).max())


def test_magnetic_gradient_finite_differences():
    m = syn.small_case(syn.SPIN, cells=(2, 2, 3), nsite=2, nmodels=1, seed=53)
    t = syn.small_case(syn.SPIN, cells=(2, 2, 3), nsite=2, nmodels=1, seed=54)
    hkl = np.random.default_rng(2).uniform(-2, 2, (30, 3))
    hkl[0] = 0.0
    target = core.magnetic_intensity_direct(t, hkl, core.TOTAL)
    chi2, grad = adjoint.magnetic_chi2_grad(m, hkl, target)
    fun = lambda: float(np.sum((core.magnetic_intensity_direct(m, hkl, core.TOTAL) - target) ** 2))
    for idx in [(0, 0, 0, 0, 0, 0), (0, 1, 1, 1, 2, 2), (0, 1, 0, 1, 1, 1)]:
        fd = _fd(fun, m, "spins", idx)
        assert math.isclose(grad[idx], fd, rel_tol=2e-5, abs_tol=1e-7 * np.abs(grad).max())


def test_oracle_uses_threads():
    assert core.oracle_threads() >= 1
    assert oracle.TOTAL == 0 and oracle.DIFFUSE == 1
