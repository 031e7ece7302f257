"""Seeded synthetic supercell models: the INPUTS that the CPU oracle and the GPU path both read.

This module holds random draws and crystal geometry (site lists, lattice constants, form-factor
coefficients) and nothing of the scattering calculation itself: no Fourier transform, no phase
factor, no intensity.  Both sides of every parity test take their inputs from here; neither side
takes anything else from the other.

The workloads mirror the shapes of the paper's examples (Section IV: pyrochlore ice-rules
supercells of ~10^3 cells carrying occupational, magnetic or displacive disorder, ~10^4-10^7
reciprocal-space points), since the paper's own Monte-Carlo supercells are not available:

* ``displacive_fcc``     fcc, a = 4 A, 4 sites, i.i.d. Gaussian displacements, f = 1
* ``pyrochlore_occ_mag`` cubic a = 10 A, 16 pyrochlore sites, Bernoulli occupancies and
                         von Mises-Fisher unit spins around seeded local axes, <j0> form factor
* ``perovskite_correlated`` cubic a = 4 A, 5 sites, Gaussian-filtered correlated displacements,
                         4-Gaussian X-ray-like form factors with seeded coefficients
* ``pyrochlore_mag_disp`` the magnetic pyrochlore whose atoms also carry Gaussian displacements
* ``serving_mix``        Poisson arrivals of mixed supercell sizes / disorder types
* ``random_origins``, ``covering_origins``  seeded sub-box origins (model, o1, o2, o3)

Array layouts (C order): occupancy uint8 [model][site][n1][n2][n3]; spins and displacements
float32 [model][site][n1][n2][n3][3] (Cartesian; spins in Bohr magnetons, displacements in
Angstrom).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

# form-factor kinds (same integer codes as the C boundary)
FF_CONST, FF_GAUSS4, FF_J0 = 0, 1, 2
# disorder kinds
OCC, SPIN, DISP = 0, 1, 2

FCC_SITES = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])

# pyrochlore lattice: fcc translations x 4-vertex tetrahedral basis (16 sites per cubic cell)
_FCC_T = FCC_SITES
_TET = np.array([[0.0, 0.0, 0.0], [0.0, 0.25, 0.25], [0.25, 0.0, 0.25], [0.25, 0.25, 0.0]])
PYROCHLORE_SITES = np.array([(t + b) % 1.0 for t in _FCC_T for b in _TET])

PEROVSKITE_SITES = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5], [0.5, 0.5, 0.0],
                             [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])

# <j0> coefficients of the magnetic workload (A, a, B, b, C, c, D)
J0_COEF = (0.4, 15.0, 0.6, 5.0, 0.0, 1.0, 0.0)


@dataclass
class QGrid:
    """Reciprocal-space grid in r.l.u.: voxel (i, j, l) <-> h0 + (i, j, l) * step, l fastest."""
    h0: Tuple[float, float, float]
    step: Tuple[float, float, float]
    count: Tuple[int, int, int]

    @property
    def nvox(self) -> int:
        return int(np.prod(self.count))

    def hkl(self) -> np.ndarray:
        """All grid points as a [nvox, 3] float64 array (r.l.u.), C order."""
        axes = [self.h0[a] + self.step[a] * np.arange(self.count[a]) for a in range(3)]
        g = np.meshgrid(*axes, indexing="ij")
        return np.stack([x.reshape(-1) for x in g], axis=1)

    def g_index(self, cells) -> np.ndarray:
        """Grid points as integer supercell Bragg indices G_alpha = n_alpha * h_alpha."""
        return np.rint(self.hkl() * np.asarray(cells, dtype=np.float64)).astype(np.int64)


@dataclass
class Model:
    """One ensemble of supercells sharing lattice, sites and supercell size."""
    lattice: Tuple[float, float, float, float, float, float]   # a, b, c (A), alpha, beta, gamma (deg)
    sites: np.ndarray                                            # [nsite, 3] fractional
    scat_len: np.ndarray                                         # [nsite]
    ff_kind: np.ndarray                                          # [nsite] int
    ff_coef: np.ndarray                                          # [nsite, 9]
    cells: Tuple[int, int, int]
    nmodels: int = 1
    occ: Optional[np.ndarray] = None
    spins: Optional[np.ndarray] = None
    disp: Optional[np.ndarray] = None
    mean_occ: Optional[np.ndarray] = None                        # None -> sample mean
    qgrid: Optional[QGrid] = None
    meta: dict = field(default_factory=dict)

    @property
    def nsite(self) -> int:
        return int(self.sites.shape[0])

    @property
    def ncell(self) -> int:
        return int(np.prod(self.cells))

    @property
    def natom(self) -> int:
        return self.nsite * self.ncell


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _ff(nsite, kind=FF_CONST, coef=None):
    kinds = np.full(nsite, kind, dtype=np.int32)
    c = np.zeros((nsite, 9))
    if coef is not None:
        c[:, :len(coef)] = np.asarray(coef, dtype=np.float64)
    return kinds, c


def symmetric_qgrid(hmax: float, cells, per_cell_step: int = 1) -> QGrid:
    """|h|,|k|,|l| <= hmax on the commensurate grid of step 1/(n_alpha) (times per_cell_step)."""
    step = tuple(per_cell_step / float(n) for n in cells)
    count = tuple(int(round(2 * hmax / s)) + 1 for s in step)
    return QGrid(h0=(-hmax, -hmax, -hmax), step=step, count=count)


def gaussian_displacements(rng, nmodels, nsite, cells, sigma) -> np.ndarray:
    return (rng.standard_normal((nmodels, nsite) + tuple(cells) + (3,)) * sigma).astype(np.float32)


def periodic_gaussian_filter(x: np.ndarray, sigma_cells: float, axes=(2, 3, 4)) -> np.ndarray:
    """Separable periodic Gaussian smoothing by direct circular convolution (np.roll sums)."""
    radius = int(np.ceil(4 * sigma_cells))
    taps = np.arange(-radius, radius + 1)
    w = np.exp(-0.5 * (taps / sigma_cells) ** 2)
    w /= w.sum()
    y = x.astype(np.float64)
    for ax in axes:
        acc = np.zeros_like(y)
        for t, wt in zip(taps, w):
            acc += wt * np.roll(y, int(t), axis=ax)
        y = acc
    return y


def correlated_displacements(rng, nmodels, nsite, cells, rms, sigma_cells) -> np.ndarray:
    """White noise smoothed by a periodic Gaussian (sigma in cells), rescaled to `rms` per component."""
    white = rng.standard_normal((nmodels, nsite) + tuple(cells) + (3,))
    y = periodic_gaussian_filter(white, sigma_cells)
    cur = np.sqrt(np.mean(y ** 2, axis=(0, 1, 2, 3, 4), keepdims=True))
    return (y * (rms / cur)).astype(np.float32)


def bernoulli_occupancy(rng, nmodels, nsite, cells, c) -> np.ndarray:
    return (rng.random((nmodels, nsite) + tuple(cells)) < c).astype(np.uint8)


def unit_vectors(rng, n) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def von_mises_fisher_spins(rng, axes: np.ndarray, kappa: float, nmodels, cells) -> np.ndarray:
    """Unit spins ~ vMF(mean axis of each site, kappa) by Wood's (1994) exact 3D sampler."""
    nsite = axes.shape[0]
    shape = (nmodels, nsite) + tuple(cells)
    xi = rng.random(shape)
    w = 1.0 + np.log(xi + (1.0 - xi) * np.exp(-2.0 * kappa)) / kappa
    w = np.clip(w, -1.0, 1.0)
    # random direction perpendicular to each site's axis
    v = rng.standard_normal(shape + (3,))
    mu = axes[None, :, None, None, None, :]
    v = v - np.sum(v * mu, axis=-1, keepdims=True) * mu
    v /= np.linalg.norm(v, axis=-1, keepdims=True)
    s = w[..., None] * mu + np.sqrt(1.0 - w ** 2)[..., None] * v
    return s.astype(np.float32)


# ----------------------------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------------------------

def displacive_fcc(cells=(8, 8, 8), sigma=0.1, seed=1, nmodels=1, hrange=(-4.0, 4.0),
                   qcount=None) -> Model:
    """fcc a = 4 A, 4 sites, i.i.d. Gaussian displacements (sigma per Cartesian component), f = 1.

    Default Q grid: h, k, l in [hrange) with step 1/n (64^3 voxels for 8^3 cells)."""
    rng = _rng(seed)
    kinds, coef = _ff(4)
    m = Model(lattice=(4.0, 4.0, 4.0, 90.0, 90.0, 90.0), sites=FCC_SITES.copy(),
              scat_len=np.ones(4), ff_kind=kinds, ff_coef=coef, cells=tuple(cells), nmodels=nmodels)
    m.disp = gaussian_displacements(rng, nmodels, 4, cells, sigma)
    step = tuple(1.0 / n for n in cells)
    if qcount is None:
        qcount = tuple(int(round((hrange[1] - hrange[0]) * n)) for n in cells)
    m.qgrid = QGrid(h0=(hrange[0],) * 3, step=step, count=tuple(qcount))
    m.meta = dict(kind="displacive", sigma=sigma, seed=seed)
    return m


def pyrochlore_occ_mag(cells=(20, 20, 20), c=0.3, kappa=2.0, seed=2, nmodels=1, hmax=6.0,
                       nsite=16) -> Model:
    """Cubic a = 10 A with the 16 pyrochlore sites; Bernoulli(c) occupancies (b = 1) and unit
    spins from vMF(kappa) around one seeded axis per site; <j0> magnetic form factor.

    The same Model carries both the occupancies (nuclear volume) and the spins (magnetic
    volume).  `nsite` < 16 keeps the first sites (smaller test cases)."""
    rng = _rng(seed)
    sites = PYROCHLORE_SITES[:nsite].copy()
    kinds, coef = _ff(nsite)
    m = Model(lattice=(10.0, 10.0, 10.0, 90.0, 90.0, 90.0), sites=sites,
              scat_len=np.ones(nsite), ff_kind=kinds, ff_coef=coef, cells=tuple(cells),
              nmodels=nmodels)
    m.occ = bernoulli_occupancy(rng, nmodels, nsite, cells, c)
    axes = unit_vectors(rng, nsite)
    m.spins = von_mises_fisher_spins(rng, axes, kappa, nmodels, cells)
    m.qgrid = symmetric_qgrid(hmax, cells)
    m.meta = dict(kind="occ+mag", c=c, kappa=kappa, seed=seed, spin_axes=axes,
                  mag_ff_kind=FF_J0, mag_ff_coef=np.array(J0_COEF + (0.0, 0.0)))
    return m


def magnetic_view(m: Model) -> Model:
    """The same supercells with the <j0> form factor on every site (for the magnetic volume)."""
    kinds = np.full(m.nsite, FF_J0, dtype=np.int32)
    coef = np.tile(np.asarray(m.meta["mag_ff_coef"], dtype=np.float64), (m.nsite, 1))
    return Model(lattice=m.lattice, sites=m.sites, scat_len=np.ones(m.nsite), ff_kind=kinds,
                 ff_coef=coef, cells=m.cells, nmodels=m.nmodels, spins=m.spins, qgrid=m.qgrid,
                 meta=dict(m.meta))


def pyrochlore_mag_disp(cells=(20, 20, 20), kappa=2.0, sigma=0.05, seed=6, nmodels=1,
                        hmax=6.0, nsite=16) -> Model:
    """The magnetic pyrochlore (<j0> on every site, vMF spins) whose atoms also carry i.i.d.
    Gaussian displacements (sigma per Cartesian component, Angstrom): the input of the
    magnetic + displacive coupling through the Debye-Waller factor."""
    m = magnetic_view(pyrochlore_occ_mag(cells=cells, kappa=kappa, seed=seed, nmodels=nmodels,
                                         hmax=hmax, nsite=nsite))
    m.disp = gaussian_displacements(_rng(seed + 500), nmodels, nsite, cells, sigma)
    m.meta["kind"] = "mag+disp"
    m.meta["sigma"] = sigma
    return m


def random_origins(rng, nmodels, cells, count) -> np.ndarray:
    """`count` sub-box origins (model, o1, o2, o3), int32, uniform over the lattice points of
    the ensemble."""
    out = np.empty((count, 4), dtype=np.int32)
    out[:, 0] = rng.integers(0, nmodels, count)
    for a in range(3):
        out[:, 1 + a] = rng.integers(0, cells[a], count)
    return out


def covering_origins(rng, nmodels, cells, nsb) -> np.ndarray:
    """Random sub-box origins, drawn per supercell until each of its lattice points lies in at
    least one box of nsb^3 cells (periodic wrap): the random-origin variant of the method of
    sub-boxes (Section V A), whose count is set by that coverage rule."""
    rows = []
    span = np.arange(nsb)
    for m in range(nmodels):
        covered = np.zeros(cells, dtype=bool)
        while not covered.all():
            o = [int(rng.integers(0, c)) for c in cells]
            idx = [np.mod(o[a] + span, cells[a]) for a in range(3)]
            covered[np.ix_(*idx)] = True
            rows.append((m, *o))
    return np.asarray(rows, dtype=np.int32)


def random_gauss4(rng, nsite) -> np.ndarray:
    """Seeded 4-Gaussian coefficients: a_i in [0.5, 10], b_i in [0.5, 50], c in [0, 2]."""
    coef = np.zeros((nsite, 9))
    coef[:, 0:4] = rng.uniform(0.5, 10.0, (nsite, 4))
    coef[:, 4:8] = rng.uniform(0.5, 50.0, (nsite, 4))
    coef[:, 8] = rng.uniform(0.0, 2.0, nsite)
    return coef


def perovskite_correlated(cells=(64, 64, 64), rms=0.08, corr_cells=3.0, seed=3, nmodels=1,
                          hmax=8.0) -> Model:
    """Cubic perovskite a = 4 A, 5 sites, correlated displacements (periodic Gaussian filter,
    sigma = corr_cells), rescaled to `rms` A per component; seeded 4-Gaussian form factors."""
    rng = _rng(seed)
    coef = random_gauss4(rng, 5)
    m = Model(lattice=(4.0, 4.0, 4.0, 90.0, 90.0, 90.0), sites=PEROVSKITE_SITES.copy(),
              scat_len=np.ones(5), ff_kind=np.full(5, FF_GAUSS4, dtype=np.int32), ff_coef=coef,
              cells=tuple(cells), nmodels=nmodels)
    m.disp = correlated_displacements(rng, nmodels, 5, cells, rms, corr_cells)
    m.qgrid = symmetric_qgrid(hmax, cells)
    m.meta = dict(kind="displacive", rms=rms, corr_cells=corr_cells, seed=seed,
                  lanczos_m=2, lanczos_mprime=cells[0] // 8)
    return m


def differentiation_pair(cells=(32, 32, 32), seed=5, hmax=5.0):
    """(model, target): model u ~ N(0, 0.1^2) i.i.d.; target from a second seed, correlated
    (periodic Gaussian filter sigma = 2 cells) rescaled to 0.07 A rms per component."""
    model = displacive_fcc(cells=cells, sigma=0.1, seed=seed)
    model.qgrid = symmetric_qgrid(hmax, cells)
    rng = _rng(seed + 1000)
    target = displacive_fcc(cells=cells, sigma=0.07, seed=seed + 1000)
    target.disp = correlated_displacements(rng, 1, 4, cells, 0.07, 2.0)
    target.qgrid = model.qgrid
    return model, target


def small_case(kind: int, cells=(6, 5, 4), nsite=3, nmodels=2, seed=11, sigma=0.05,
               qgrid: Optional[QGrid] = None) -> Model:
    """Tiny mixed-geometry case (triclinic lattice, arbitrary sites, mixed form factors) for
    parity tests that span several tiles with ragged tails."""
    rng = _rng(seed)
    sites = rng.random((nsite, 3))
    kinds = np.array([(FF_CONST, FF_GAUSS4, FF_J0)[i % 3] for i in range(nsite)], dtype=np.int32)
    coef = np.zeros((nsite, 9))
    g4 = random_gauss4(rng, nsite)
    for i in range(nsite):
        if kinds[i] == FF_GAUSS4:
            coef[i] = g4[i]
        elif kinds[i] == FF_J0:
            coef[i, :7] = J0_COEF
    m = Model(lattice=(4.1, 4.6, 5.2, 84.0, 97.0, 101.0), sites=sites,
              scat_len=rng.uniform(0.5, 2.0, nsite), ff_kind=kinds, ff_coef=coef,
              cells=tuple(cells), nmodels=nmodels)
    if kind == OCC:
        m.occ = bernoulli_occupancy(rng, nmodels, nsite, cells, 0.4)
    elif kind == SPIN:
        m.spins = von_mises_fisher_spins(rng, unit_vectors(rng, nsite), 1.5, nmodels, cells)
    else:
        m.disp = gaussian_displacements(rng, nmodels, nsite, cells, sigma)
        if nsite > 1:
            m.occ = bernoulli_occupancy(rng, nmodels, nsite, cells, 0.7)
    if qgrid is None:
        qgrid = QGrid(h0=tuple(-1.0 - 2.0 / n for n in cells), step=tuple(1.0 / n for n in cells),
                      count=tuple(2 * n + 3 for n in cells))
    m.qgrid = qgrid
    m.meta = dict(kind=("occ", "spin", "disp")[kind], seed=seed)
    return m


def serving_mix(nreq=512, seed=4, rate_hz=200.0, sizes=(16, 32, 48, 64), hmax=4.0,
                max_nsite=16):
    """Request stream: Poisson arrival times (seconds) and a request spec per arrival."""
    rng = _rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, nreq))
    reqs = []
    for i in range(nreq):
        n = int(rng.choice(sizes))
        kind = int(rng.integers(0, 3))
        nsite = int(rng.integers(1, max_nsite + 1))
        reqs.append(dict(arrival=float(t[i]), n=n, kind=kind, nsite=nsite,
                         seed=int(rng.integers(0, 2 ** 31)), hmax=hmax))
    return reqs


def serving_model(spec) -> Model:
    """Materialise one serving request spec into a Model."""
    rng = _rng(spec["seed"])
    n, nsite, kind = spec["n"], spec["nsite"], spec["kind"]
    cells = (n, n, n)
    sites = rng.random((nsite, 3))
    kinds, coef = _ff(nsite)
    m = Model(lattice=(5.0, 5.0, 5.0, 90.0, 90.0, 90.0), sites=sites, scat_len=np.ones(nsite),
              ff_kind=kinds, ff_coef=coef, cells=cells, nmodels=1)
    if kind == OCC:
        m.occ = bernoulli_occupancy(rng, 1, nsite, cells, 0.3)
    elif kind == SPIN:
        m.spins = von_mises_fisher_spins(rng, unit_vectors(rng, nsite), 2.0, 1, cells)
        m.ff_kind[:] = FF_J0
        m.ff_coef[:, :7] = J0_COEF
    else:
        m.disp = gaussian_displacements(rng, 1, nsite, cells, 0.03)
    m.qgrid = symmetric_qgrid(spec["hmax"], cells)
    m.meta = dict(kind=("occ", "spin", "disp")[kind])
    return m
