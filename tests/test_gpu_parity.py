"""GPU path vs the CPU FP64 oracle, element by element, through the C boundary.

Tolerances (max |I_gpu - I_oracle| / max |I_oracle|): 1e-10 for the FP64 path, 1e-5 for the
FP32 path.  The displacive path additionally differs from the exact direct sum by at most the
Taylor remainder bound of Section III C.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import core, noise
from _helpers import TOL, qgrid_tuple, rel_err_of_peak, to_library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1809_07088_gb300 as ds
    c = ds.Context(0)
    yield c
    c.close()


def _G(m):
    return m.qgrid.g_index(m.cells)


PREC = [(0, "fp64"), (1, "fp32")]


@pytest.mark.parametrize("prec,tag", PREC)
@pytest.mark.parametrize("mode", [0, 1])
def test_occupancy_small_triclinic(ctx, prec, tag, mode):
    m = syn.small_case(syn.OCC, cells=(6, 5, 4), nsite=3, nmodels=2, seed=101)
    lm = to_library(ctx, m)
    got, info = lm.intensity(qgrid_tuple(m.qgrid), disorder=0, mode=mode, precision=prec)
    want = core.occupancy_intensity_fft(m, _G(m), mode)
    assert rel_err_of_peak(got, want) < TOL[tag]
    direct = core.occupancy_intensity_direct(m, m.qgrid.hkl(), mode)
    assert rel_err_of_peak(got, direct) < TOL[tag]
    assert info["nvox"] == m.qgrid.nvox


@pytest.mark.parametrize("prec,tag", PREC)
@pytest.mark.parametrize("mode", [0, 1])
def test_magnetic_small_triclinic(ctx, prec, tag, mode):
    m = syn.small_case(syn.SPIN, cells=(5, 6, 6), nsite=4, nmodels=2, seed=102)
    assert np.any(np.all(_G(m) == 0, axis=1))       # includes Q = 0
    lm = to_library(ctx, m)
    got, _ = lm.intensity(qgrid_tuple(m.qgrid), disorder=1, mode=mode, precision=prec)
    want = core.magnetic_intensity_fft(m, _G(m), mode)
    assert rel_err_of_peak(got, want) < TOL[tag]


KERNELS = [1, 2]   # the per-voxel and the sum-factorised evaluation of the Taylor sum


@pytest.mark.parametrize("kern", KERNELS)
@pytest.mark.parametrize("prec,tag", PREC)
@pytest.mark.parametrize("mode", [0, 1])
def test_displacive_small_with_occupancy(ctx, prec, tag, mode, kern):
    m = syn.small_case(syn.DISP, cells=(4, 6, 5), nsite=3, nmodels=2, seed=103, sigma=0.05)
    lm = to_library(ctx, m)
    P = 7
    got, info = lm.intensity(qgrid_tuple(m.qgrid), disorder=2, mode=mode, precision=prec, taylor_order=P,
                             taylor_kernel=kern)
    assert info["taylor_order"] == P and info["n_monomials"] == (P + 1) * (P + 2) * (P + 3) // 6
    want = core.displacive_intensity_fft(m, _G(m), mode, P=P)
    assert rel_err_of_peak(got, want) < TOL[tag]
    hkl = m.qgrid.hkl()
    I_dir, F = core.displacive_intensity_direct(m, hkl, mode, return_F=True)
    bound = core.truncation_bound(m, hkl, P, mode, F=F)
    peak = np.max(np.abs(I_dir))
    assert np.all(np.abs(got.reshape(-1) - I_dir) <= bound + 2 * TOL[tag] * peak)


@pytest.mark.parametrize("prec,tag", PREC)
@pytest.mark.parametrize("mode", [0, 1])
def test_displacive_zone_orders_small(ctx, prec, tag, mode):
    """Per-zone Taylor orders (taylor_zonal = 1): voxel by voxel equal to the oracle's zone-order
    method, within the per-voxel remainder bound of the direct sum; the served request gives
    the same bits."""
    import torch
    m = syn.small_case(syn.DISP, cells=(4, 6, 5), nsite=3, nmodels=2, seed=105, sigma=0.15)
    lm = to_library(ctx, m)
    q = qgrid_tuple(m.qgrid)
    opts = dict(disorder=2, mode=mode, precision=prec, taylor_order=-1, taylor_eps=1e-6, taylor_zonal=1)
    got, info = lm.intensity(q, **opts)
    pv, P = core.zone_taylor_orders(m, m.qgrid, 1e-6)
    assert info["taylor_order"] == P and len(np.unique(pv)) >= 2
    want = core.displacive_intensity_fft(m, _G(m), mode, P=P, P_vox=pv)
    assert rel_err_of_peak(got, want) < TOL[tag]
    hkl = m.qgrid.hkl()
    I_dir, F = core.displacive_intensity_direct(m, hkl, mode, return_F=True)
    bound = core.truncation_bound(m, hkl, pv, mode, F=F)
    assert np.all(np.abs(got.reshape(-1) - I_dir) <= bound + 2 * TOL[tag] * np.max(np.abs(I_dir)))
    out = torch.empty(m.qgrid.count, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    t = lm.submit(q, out, **opts)
    ctx.wait(t, 60.0)
    assert np.array_equal(out.cpu().numpy(), got)


@pytest.mark.parametrize("prec,tag", PREC)
def test_displacive_fcc_8cubed_zone_orders_full_volume(ctx, prec, tag):
    """fcc 8^3, 64^3 voxels, per-zone orders at eps = 1e-8: the whole volume within the
    per-voxel remainder bound of the exact direct sum; sampled voxels (Bragg positions
    included) against the oracle's zone-order method."""
    m = syn.displacive_fcc()
    lm = to_library(ctx, m)
    got, info = lm.intensity(qgrid_tuple(m.qgrid), disorder=2, mode=1, precision=prec, taylor_order=-1,
                             taylor_eps=1e-8, taylor_zonal=1)
    pv, P = core.zone_taylor_orders(m, m.qgrid, 1e-8)
    assert info["taylor_order"] == P and pv.min() < P
    hkl = m.qgrid.hkl()
    I_dir, F = core.displacive_intensity_direct(m, hkl, 1, return_F=True)
    bound = core.truncation_bound(m, hkl, pv, 1, F=F)
    peak = np.max(I_dir)
    assert np.all(np.abs(got.reshape(-1) - I_dir) <= bound + TOL[tag] * peak)
    rng = np.random.default_rng(1)
    G = _G(m)
    idx = np.concatenate([rng.choice(G.shape[0], 400, replace=False),
                          np.nonzero(np.all(np.mod(G, 8) == 0, axis=1))[0][:40]])
    want = core.displacive_intensity_fft(m, G[idx], 1, P=P, P_vox=pv[idx])
    assert np.max(np.abs(got.reshape(-1)[idx] - want)) < TOL[tag] * peak


@pytest.mark.parametrize("cells", [(7, 9, 10), (12, 5, 8), (3, 14, 6), (16, 16, 16), (1, 1, 2), (2, 3, 1)])
def test_fft_sizes_all_radices(ctx, cells):
    """Supercells with factors 2, 3, 4, 5, 7 and degenerate axes, FP64 parity."""
    m = syn.small_case(syn.OCC, cells=cells, nsite=2, nmodels=1, seed=104)
    lm = to_library(ctx, m)
    got, _ = lm.intensity(qgrid_tuple(m.qgrid), disorder=0, mode=0, precision=0)
    want = core.occupancy_intensity_fft(m, _G(m), 0)
    assert rel_err_of_peak(got, want) < TOL["fp64"]


@pytest.mark.parametrize("n", [8, 16, 20, 32, 64])
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_fft_register_kernel_cubic_sizes(ctx, n, kind):
    """Cubic FP32 supercells of 8, 16, 20 and 32 cells (one CTA per field, lines in registers) and of
    64 cells (planes, then columns, each 64-point line split over eight threads): occupancy, moments
    and Taylor monomials (the i^n factor of every order), two supercells, against the oracle's FFT
    method."""
    q = syn.QGrid(h0=(-1.0 - 2.0 / n,) * 3, step=(1.0 / n,) * 3, count=(n + 5, n + 3, 2 * n + 1))
    m = syn.small_case(kind, cells=(n, n, n), nsite=2, nmodels=2, seed=600 + n + kind, qgrid=q)
    lm = to_library(ctx, m)
    G = _G(m)
    if kind == 2:
        got, _ = lm.intensity(qgrid_tuple(q), disorder=2, mode=1, precision=1, taylor_order=5)
        want = core.displacive_intensity_fft(m, G, 1, P=5)
    elif kind == 1:
        got, _ = lm.intensity(qgrid_tuple(q), disorder=1, mode=0, precision=1)
        want = core.magnetic_intensity_fft(m, G, 0)
    else:
        got, _ = lm.intensity(qgrid_tuple(q), disorder=0, mode=1, precision=1)
        want = core.occupancy_intensity_fft(m, G, 1)
    assert rel_err_of_peak(got, want) < TOL["fp32"]


@pytest.mark.parametrize("prec,tag", PREC)
def test_fft_two_pass_radices(ctx, prec, tag):
    """A supercell too large for the whole-field FFT kernel (30 x 28 x 35: radices 2, 3, 4, 5, 7)
    goes through the two-pass plane/column FFT; parity with the oracle."""
    m = syn.small_case(syn.OCC, cells=(30, 28, 35), nsite=2, nmodels=1, seed=105)
    lm = to_library(ctx, m)
    got, _ = lm.intensity(qgrid_tuple(m.qgrid), disorder=0, mode=1, precision=prec)
    assert rel_err_of_peak(got, core.occupancy_intensity_fft(m, _G(m), 1)) < TOL[tag]


def test_single_voxel_and_single_zone_grids(ctx):
    m = syn.small_case(syn.SPIN, cells=(4, 4, 4), nsite=2, nmodels=1, seed=105)
    lm = to_library(ctx, m)
    for q in [syn.QGrid((0.25, -0.5, 1.0), (0.25,) * 3, (1, 1, 1)),
              syn.QGrid((1.0, 2.0, -1.0), (0.25,) * 3, (4, 4, 4)),
              syn.QGrid((0.0, 0.0, 0.0), (0.25,) * 3, (1, 1, 1))]:
        got, _ = lm.intensity(qgrid_tuple(q), disorder=1, mode=0, precision=0)
        want = core.magnetic_intensity_fft(m, q.g_index(m.cells), 0)
        assert rel_err_of_peak(got, want) < TOL["fp64"]


@pytest.mark.parametrize("m_,mp", [(2, 2), (3, 2), (2, 4)])
def test_lanczos_commensurate(ctx, m_, mp):
    """Section V B on the commensurate grid: GPU stencil vs the literal finite sum of Eq.
    intensity_convol_finite, with I(G) from the oracle's FFT method (halo included)."""
    m = syn.small_case(syn.OCC, cells=(6, 5, 4), nsite=3, nmodels=1, seed=106)
    lm = to_library(ctx, m)
    for prec, tag in PREC:
        got, _ = lm.intensity(qgrid_tuple(m.qgrid), disorder=0, mode=1, precision=prec, smoothing=1,
                              lanczos_m=m_, lanczos_mprime=mp)
        IG = lambda G: core.occupancy_intensity_fft(m, G, 1)
        want = noise.lanczos_resample(IG, _G(m).astype(np.float64), m_, mp)
        assert rel_err_of_peak(got, want) < TOL[tag]


@pytest.mark.parametrize("prec,tag", PREC)
@pytest.mark.parametrize("m_,mp", [(2, 2), (3, 2), (2, 4)])
def test_points_arbitrary_occupancy(ctx, prec, tag, m_, mp):
    """Lanczos resampling at arbitrary wavevectors (Section V B, Eq. intensity_convol_finite with
    floor bounds and the strict window): random points, points on Bragg positions and negative
    coordinates, against the oracle's literal finite sum over I(G) of the oracle's FFT method."""
    m = syn.small_case(syn.OCC, cells=(6, 5, 4), nsite=3, nmodels=2, seed=131)
    lm = to_library(ctx, m)
    rng = np.random.default_rng(7)
    hkl = np.concatenate([rng.uniform(-1.3, 1.3, (200, 3)),
                          np.array([[0.0, 0.0, 0.0], [1 / 6, -2 / 5, 0.25], [-1.0, 0.5, 1.0]])])
    got, info = lm.intensity_points(hkl, disorder=0, mode=1, precision=prec, lanczos_m=m_, lanczos_mprime=mp)
    assert info["nvox"] == hkl.shape[0]
    Q = hkl * np.array(m.cells)
    want = noise.lanczos_resample(lambda G: core.occupancy_intensity_fft(m, G, 1), Q, m_, mp)
    assert rel_err_of_peak(got, want) < TOL[tag]


@pytest.mark.parametrize("prec,tag", PREC)
def test_points_hhl_plane_magnetic(ctx, prec, tag):
    """An (h h l) plane off the Bragg grid (the paper's plane geometry, Section IV) for the
    magnetic intensity with the <j0> form factor, device points and device output."""
    import torch
    m = syn.pyrochlore_occ_mag(cells=(4, 4, 4), nmodels=2, hmax=1.0, seed=12)
    mm = syn.magnetic_view(m)
    lm = to_library(ctx, mm)
    u, v = np.meshgrid(np.linspace(-1.55, 1.45, 23), np.linspace(-2.1, 1.9, 21), indexing="ij")
    hkl = np.stack([u.ravel(), u.ravel(), v.ravel()], axis=1)
    dt = torch.float64 if prec == 0 else torch.float32
    out = torch.empty(hkl.shape[0], dtype=dt, device="cuda")
    lm.intensity_points(torch.from_numpy(hkl).cuda(), out=out, disorder=1, mode=0, precision=prec, lanczos_m=2,
                        lanczos_mprime=2)
    torch.cuda.synchronize()
    want = noise.lanczos_resample(lambda G: core.magnetic_intensity_fft(mm, G, 0), hkl * 4.0, 2, 2)
    assert rel_err_of_peak(out.cpu().numpy(), want) < TOL[tag]


@pytest.mark.parametrize("prec,tag", PREC)
def test_points_displacive_and_grid_consistency(ctx, prec, tag):
    """Displacive points (fixed Taylor order) against the oracle; points placed exactly on Bragg
    positions equal the commensurate Lanczos volume of ds_request_intensity."""
    m = syn.small_case(syn.DISP, cells=(4, 6, 5), nsite=3, nmodels=2, seed=132, sigma=0.08)
    lm = to_library(ctx, m)
    rng = np.random.default_rng(8)
    hkl = rng.uniform(-0.9, 0.9, (120, 3))
    opts = dict(disorder=2, mode=1, precision=prec, taylor_order=6, lanczos_m=2, lanczos_mprime=2)
    got, _ = lm.intensity_points(hkl, **opts)
    want = noise.lanczos_resample(lambda G: core.displacive_intensity_fft(m, G, 1, P=6), hkl * np.array(m.cells), 2, 2)
    assert rel_err_of_peak(got, want) < TOL[tag]
    vol, _ = lm.intensity(qgrid_tuple(m.qgrid), smoothing=1, **opts)
    G = _G(m)
    pick = np.random.default_rng(9).choice(G.shape[0], 50, replace=False)
    on_grid, _ = lm.intensity_points(G[pick] / np.array(m.cells), **opts)
    assert rel_err_of_peak(on_grid, vol.reshape(-1)[pick]) < TOL[tag]


def test_points_errors(ctx):
    import paper_1809_07088_gb300 as ds
    m = syn.small_case(syn.OCC, cells=(3, 3, 3), nsite=1, nmodels=1, seed=133)
    lm = to_library(ctx, m)
    with pytest.raises(ds.DSError):
        lm.intensity_points(np.zeros((3, 3)), disorder=0, smoothing=0)
    with pytest.raises(ds.DSError):
        lm.intensity_points(np.array([[np.nan, 0.0, 0.0]]), disorder=0)
    out, info = lm.intensity_points(np.zeros((0, 3)), disorder=0)
    assert out.shape == (0,) and info["nvox"] == 0


def test_points_checked_on_the_device(ctx):
    """Points given on the device are scaled and bounded there: the first non-finite point is
    reported by its index (here the 2nd of three in a block of 300, and again past the first
    block of the reduction), points whose box of Bragg positions would be too long along an axis
    are refused, and a valid device request matches the same request from host memory bit for
    bit."""
    import torch
    import paper_1809_07088_gb300 as ds
    m = syn.small_case(syn.OCC, cells=(3, 3, 3), nsite=1, nmodels=1, seed=134)
    lm = to_library(ctx, m)
    rng = np.random.default_rng(5)
    for bad_at in (151, 1000):
        hkl = rng.uniform(-1.0, 1.0, (1200, 3))
        hkl[bad_at, 1] = np.inf
        hkl[bad_at + 7, 0] = np.nan
        with pytest.raises(ds.DSError) as e:
            lm.intensity_points(torch.from_numpy(hkl).cuda(), out=torch.empty(1200, device="cuda"),
                                disorder=0, precision=1)
        assert "DS_ERR_ARG" in str(e.value) and ("point %d is not finite" % bad_at) in str(e.value)
    far = np.array([[0.0, 0.0, 0.0], [0.0, 2.0e6, 0.0]])
    with pytest.raises(ds.DSError) as e:
        lm.intensity_points(torch.from_numpy(far).cuda(), out=torch.empty(2, device="cuda"), disorder=0,
                            precision=1)
    assert "DS_ERR_UNSUPPORTED" in str(e.value) and "axis 1" in str(e.value)
    hkl = rng.uniform(-1.2, 1.1, (777, 3))
    host, _ = lm.intensity_points(hkl, disorder=0, mode=1, precision=1)
    dev = torch.empty(777, dtype=torch.float32, device="cuda")
    lm.intensity_points(torch.from_numpy(hkl).cuda(), out=dev, disorder=0, mode=1, precision=1)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), host)


@pytest.mark.parametrize("prec,tag", PREC)
@pytest.mark.parametrize("m_,mp", [(2, 2), (3, 2), (2, 4), (3, 3)])
def test_sphere_cutoff_commensurate_and_points(ctx, prec, tag, m_, mp):
    """Spherically symmetric cutoff W_r(|Q - G|) with the Lanczos window (Section V B): on the grid
    of Bragg positions (3D stencil) and at arbitrary points, triclinic cell, against the oracle's
    literal finite sum."""
    m = syn.small_case(syn.OCC, cells=(6, 5, 4), nsite=3, nmodels=2, seed=141)
    lm = to_library(ctx, m)
    I_at = lambda G: core.occupancy_intensity_fft(m, G, 1)
    got, _ = lm.intensity(qgrid_tuple(m.qgrid), disorder=0, mode=1, precision=prec, smoothing=3, lanczos_m=m_,
                          lanczos_mprime=mp)
    want = noise.sphere_resample(m, I_at, _G(m).astype(float), m_, mp)
    assert rel_err_of_peak(got, want) < TOL[tag]
    hkl = np.random.default_rng(12).uniform(-1.2, 1.2, (150, 3))
    gp, _ = lm.intensity_points(hkl, disorder=0, mode=1, precision=prec, smoothing=3, lanczos_m=m_,
                                lanczos_mprime=mp)
    assert rel_err_of_peak(gp, noise.sphere_resample(m, I_at, hkl * np.array(m.cells), m_, mp)) < TOL[tag]


def test_device_output_on_torch_stream(ctx):
    import torch
    m = syn.small_case(syn.OCC, cells=(6, 5, 4), nsite=3, nmodels=1, seed=107)
    lm = to_library(ctx, m)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        out = torch.empty(m.qgrid.count, dtype=torch.float32, device="cuda")
        lm.intensity(qgrid_tuple(m.qgrid), out=out, disorder=0, mode=1, precision=1)
    s.synchronize()
    want = core.occupancy_intensity_fft(m, _G(m), 1)
    assert rel_err_of_peak(out.cpu().numpy(), want) < TOL["fp32"]


def test_upload_on_one_stream_request_on_another(ctx):
    """A device upload queued on one stream behind a long kernel, then a request on another
    stream: the request waits for the upload (and the site means computed with it)."""
    import torch
    if not hasattr(torch.cuda, "_sleep"):
        pytest.skip("torch.cuda._sleep not available")
    m = syn.small_case(syn.SPIN, cells=(4, 5, 6), nsite=3, nmodels=1, seed=121)
    lm = to_library(ctx, m)
    q = qgrid_tuple(m.qgrid)
    m.spins = syn.small_case(syn.SPIN, cells=(4, 5, 6), nsite=3, nmodels=1, seed=122).spins
    new = torch.from_numpy(np.ascontiguousarray(m.spins)).cuda()
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with torch.cuda.stream(s1):
        torch.cuda._sleep(20_000_000)
        lm.upload_spins(new)
    out = torch.empty(m.qgrid.count, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(s2):
        lm.intensity(q, out=out, disorder=1, mode=1, precision=0)
    torch.cuda.synchronize()
    want = core.magnetic_intensity_fft(m, _G(m), 1)
    assert rel_err_of_peak(out.cpu().numpy(), want) < TOL["fp64"]


def test_errors_are_reported(ctx):
    import paper_1809_07088_gb300 as ds
    m = syn.small_case(syn.OCC, cells=(4, 4, 4), nsite=2, nmodels=1, seed=108)
    lm = to_library(ctx, m)
    bad = syn.QGrid((0.0, 0.0, 0.0), (0.3, 0.25, 0.25), (3, 3, 3))
    with pytest.raises(ds.DSError) as e:
        lm.intensity(qgrid_tuple(bad), disorder=0)
    assert "DS_ERR_UNSUPPORTED" in str(e.value) and "commensurate" in str(e.value)
    with pytest.raises(ds.DSError) as e:
        lm.intensity(qgrid_tuple(m.qgrid), disorder=2)
    assert "DS_ERR_STATE" in str(e.value)


def test_taylor_kernel_option_errors(ctx):
    """The Taylor-kernel choice is validated: an unknown value, the sum-factorised kernel with zone
    orders, and the sum-factorised kernel on a grid whose zone boxes are wider than 17 are refused."""
    import paper_1809_07088_gb300 as ds
    m = syn.small_case(syn.DISP, cells=(2, 2, 2), nsite=1, nmodels=1, seed=109, sigma=0.03)
    lm = to_library(ctx, m)
    q = qgrid_tuple(m.qgrid)
    with pytest.raises(ds.DSError) as e:
        lm.intensity(q, disorder=2, taylor_order=3, taylor_kernel=7)
    assert "DS_ERR_ARG" in str(e.value)
    with pytest.raises(ds.DSError) as e:
        lm.intensity(q, disorder=2, taylor_order=-1, taylor_eps=1e-6, taylor_zonal=1, taylor_kernel=2)
    assert "DS_ERR_UNSUPPORTED" in str(e.value)
    wide = ((-10.0, -10.0, -10.0), (0.5, 0.5, 0.5), (41, 5, 5))   # 21 zones along the first axis
    with pytest.raises(ds.DSError) as e:
        lm.intensity(wide, disorder=2, taylor_order=3, taylor_kernel=2)
    assert "DS_ERR_UNSUPPORTED" in str(e.value)
    got, _ = lm.intensity(wide, disorder=2, mode=0, precision=0, taylor_order=3)
    want = core.displacive_intensity_fft(m, syn.QGrid(*wide).g_index(m.cells), 0, P=3)
    assert rel_err_of_peak(got, want) < TOL["fp64"]


# ----------------------------------------------------------------------------------------------
# the workloads at full size
# ----------------------------------------------------------------------------------------------

def test_displacive_fcc_8cubed_fp64_full_volume(ctx):
    """fcc 8^3, sigma = 0.1 A, 64^3 voxels, FP64, Taylor order chosen by the remainder bound:
    the whole volume against the exact direct sum within the bound, and a voxel sample
    against the oracle's own Taylor FFT method at the same order."""
    m = syn.displacive_fcc()
    lm = to_library(ctx, m)
    got, info = lm.intensity(qgrid_tuple(m.qgrid), disorder=2, mode=1, precision=0, taylor_order=-1,
                             taylor_eps=1e-8)
    xm = core.x_max(m, m.qgrid)
    assert abs(info["x_max"] - xm) < 1e-9 * xm
    P = info["taylor_order"]
    assert P == core.taylor_order(xm, 1e-8)
    hkl = m.qgrid.hkl()
    I_dir, F = core.displacive_intensity_direct(m, hkl, 1, return_F=True)
    bound = core.truncation_bound(m, hkl, P, 1, F=F)
    peak = np.max(I_dir)
    assert np.all(np.abs(got.reshape(-1) - I_dir) <= bound + 1e-10 * peak)
    rng = np.random.default_rng(0)
    G = _G(m)
    idx = np.concatenate([rng.choice(G.shape[0], 600, replace=False),
                          np.nonzero(np.all(np.mod(G, 8) == 0, axis=1))[0][:40]])
    want = core.displacive_intensity_fft(m, G[idx], 1, P=P)
    assert rel_err_of_peak(got.reshape(-1)[idx], want) < TOL["fp64"]


def test_pyrochlore_occ_mag_20cubed(ctx):
    """16 pyrochlore sites, 20^3 cells, 241^3 voxels (the benchmark workload): FP32 within
    1e-5 of peak of the FP64 GPU path; FP64 within 1e-10 of the oracle on whole zones and on
    random voxels (direct sum)."""
    m = syn.pyrochlore_occ_mag()
    mm = syn.magnetic_view(m)
    lm_n = to_library(ctx, m, with_spins=False)
    lm_m = to_library(ctx, mm)
    q = qgrid_tuple(m.qgrid)
    G = _G(m)
    rng = np.random.default_rng(1)
    idx = rng.choice(G.shape[0], 3000, replace=False)
    H = np.floor_divide(G, 20)
    zone = np.nonzero(np.all(H == [1, -2, 0], axis=1) | np.all(H == [-6, 5, 3], axis=1))[0]
    for lm, model, dis, mode, fft in [(lm_n, m, 0, 1, core.occupancy_intensity_fft),
                                      (lm_m, mm, 1, 0, core.magnetic_intensity_fft)]:
        I64, _ = lm.intensity(q, disorder=dis, mode=mode, precision=0)
        I32, _ = lm.intensity(q, disorder=dis, mode=mode, precision=1)
        assert rel_err_of_peak(I32, I64) < 1e-5
        I64f = I64.reshape(-1)
        peak = np.max(I64f)
        want_z = fft(model, G[zone], mode)
        assert np.max(np.abs(I64f[zone] - want_z)) < 1e-10 * peak
        if dis == 0:
            want_d = core.occupancy_intensity_direct(model, G[idx] / 20.0, mode)
        else:
            want_d = core.magnetic_intensity_direct(model, G[idx] / 20.0, mode)
        assert np.max(np.abs(I64f[idx] - want_d)) < 1e-10 * peak


@pytest.mark.parametrize("dis", [0, 1])
def test_grouped_sites_several_form_factor_classes(ctx, dis):
    """Pyrochlore sites share z coordinates, so the recombination sums sites group by group;
    two form-factor classes (constant and <j0>) and two supercells, FP64 and FP32."""
    m = syn.pyrochlore_occ_mag(cells=(5, 4, 6), nmodels=2, hmax=1.0, seed=9)
    m.ff_kind = np.array([0] * 8 + [2] * 8, dtype=np.int32)
    m.ff_coef = np.zeros((16, 9))
    m.ff_coef[8:, :7] = syn.J0_COEF
    m.scat_len = np.linspace(0.5, 2.0, 16)
    lm = to_library(ctx, m)
    for prec, tag in PREC:
        got, _ = lm.intensity(qgrid_tuple(m.qgrid), disorder=dis, mode=1, precision=prec)
        fn = core.occupancy_intensity_fft if dis == 0 else core.magnetic_intensity_fft
        want = fn(m, _G(m), 1)
        assert rel_err_of_peak(got, want) < TOL[tag]


def _special_positions_case(kind, nsite, ff, seed, cells=(5, 6, 4), shift=0):
    """Sites on multiples of 1/4, 1/3 and 1/2 along the three axes (zone phases periodic in H
    with periods 4, 3, 2; suffix _xr: random first coordinates), a triclinic cell, two
    supercells and a ragged grid of 6 zones per axis, so that the residue-class recombination
    applies.  The grid is centrosymmetric (the half-grid Friedel mode) unless `shift` moves it by
    that many voxels along the last axis (an int) or along each axis (a tuple)."""
    sh = (0, 0, shift) if np.isscalar(shift) else tuple(shift)
    q = syn.QGrid(h0=tuple(-3.0 + (3.0 + s) / n for n, s in zip(cells, sh)),
                  step=tuple(1.0 / n for n in cells), count=tuple(6 * n - 5 for n in cells))
    m = syn.small_case(kind, cells=cells, nsite=nsite, nmodels=2, seed=seed, qgrid=q)
    rng = np.random.default_rng(seed)
    m.sites = np.stack([rng.integers(0, 4, nsite) / 4.0, rng.integers(0, 3, nsite) / 3.0,
                        rng.integers(0, 2, nsite) / 2.0 + rng.integers(-1, 2, nsite)], axis=1)
    if ff.endswith("_xr"):  # no period along the first axis: every zone H1 its own class
        m.sites[:, 0] = rng.random(nsite)
    if ff.startswith("one_j0"):
        m.ff_kind = np.full(nsite, syn.FF_J0, dtype=np.int32)
        m.ff_coef = np.zeros((nsite, 9))
        m.ff_coef[:, :7] = syn.J0_COEF
    elif ff == "const":
        m.ff_kind = np.zeros(nsite, dtype=np.int32)
    elif ff == "one_g4":
        m.ff_kind = np.full(nsite, syn.FF_GAUSS4, dtype=np.int32)
        m.ff_coef = np.tile(syn.random_gauss4(np.random.default_rng(seed), 1), (nsite, 1))
    return m


@pytest.mark.parametrize("prec,tag", PREC)
@pytest.mark.parametrize("disorder,ff,mode", [(0, "one_g4", 1), (1, "one_j0", 0), (1, "one_g4", 1), (0, "const", 0)])
def test_residue_classes_orthorhombic_cell(ctx, prec, tag, disorder, ff, mode):
    """Special positions in an orthorhombic cell (reciprocal axes along x, y, z): the row kernel
    factors each Gaussian of the form factor into a per-row and a per-voxel part; voxel by voxel
    equal to the oracle, Q = 0 included, two supercells accumulated."""
    m = _special_positions_case(disorder, 6, ff, 500 + disorder, cells=(5, 6, 4))
    m.lattice = (4.1, 4.6, 5.2, 90.0, 90.0, 90.0)
    G = _G(m)
    assert np.any(np.all(G == 0, axis=1))
    lm = to_library(ctx, m)
    got, _ = lm.intensity(qgrid_tuple(m.qgrid), disorder=disorder, mode=mode, precision=prec)
    fn = core.occupancy_intensity_fft if disorder == 0 else core.magnetic_intensity_fft
    assert rel_err_of_peak(got, fn(m, G, mode)) < TOL[tag]


@pytest.mark.parametrize("prec,tag", PREC)
@pytest.mark.parametrize("disorder,nsite,ff,mode", [(0, 6, "mixed", 1), (0, 20, "const", 0), (0, 5, "one_j0", 1),
                                                    (1, 6, "mixed", 0), (1, 7, "one_j0", 1), (1, 16, "const", 0),
                                                    (1, 5, "one_j0_xr", 0), (0, 4, "mixed_xr", 1)])
def test_residue_classes_special_positions(ctx, prec, tag, disorder, nsite, ff, mode):
    """Sites on special positions: the zone phases repeat with H, and the library forms the site
    sum once per residue class of zones; voxel by voxel equal to the oracle (Q = 0 included,
    one or several form-factor classes, up to 20 sites)."""
    m = _special_positions_case(disorder, nsite, ff, 200 + nsite)
    G = _G(m)
    assert np.any(np.all(G == 0, axis=1))
    lm = to_library(ctx, m)
    got, _ = lm.intensity(qgrid_tuple(m.qgrid), disorder=disorder, mode=mode, precision=prec)
    fn = core.occupancy_intensity_fft if disorder == 0 else core.magnetic_intensity_fft
    assert rel_err_of_peak(got, fn(m, G, mode)) < TOL[tag]


@pytest.mark.parametrize("prec,tag", PREC)
@pytest.mark.parametrize("cells,shift", [((5, 6, 4), 0), ((4, 6, 5), 0), ((5, 4, 7), 0), ((5, 6, 4), 1),
                                         ((4, 6, 5), -2), ((5, 6, 4), (1, -1, 0)), ((4, 6, 5), (2, 0, 1)),
                                         ((6, 5, 4), (0, 3, -1))])
@pytest.mark.parametrize("disorder,ff", [(0, "one_j0"), (1, "one_j0"), (1, "mixed")])
def test_residue_classes_centred_and_shifted_grids(ctx, prec, tag, cells, shift, disorder, ff):
    """Residue-class recombination on centrosymmetric grids with even and odd n3 and on shifted
    grids, two supercells accumulated: voxel by voxel equal to the oracle, and I(-G) = I(G)
    (Friedel symmetry of real fields) within the tolerance when the grid is centred."""
    m = _special_positions_case(disorder, 6, ff, 400 + disorder, cells=cells, shift=shift)
    lm = to_library(ctx, m)
    got, _ = lm.intensity(qgrid_tuple(m.qgrid), disorder=disorder, mode=1 - disorder, precision=prec)
    fn = core.occupancy_intensity_fft if disorder == 0 else core.magnetic_intensity_fft
    assert rel_err_of_peak(got, fn(m, _G(m), 1 - disorder)) < TOL[tag]
    if np.all(np.asarray(shift) == 0):
        assert rel_err_of_peak(got, got[::-1, ::-1, ::-1]) < TOL[tag]


@pytest.mark.parametrize("disorder,kind", [("occ", 0), ("spin", 1)])
@pytest.mark.parametrize("nsb,mode", [(1, 1), (2, 0), (3, 1)])
def test_subbox_against_brute_force(ctx, disorder, kind, nsb, mode):
    """Section V A: every lattice point the origin of an n_sb^3 open box; the GPU pair-spectrum
    route against the oracle's literal loop over origins (commensurate grid)."""
    m = syn.small_case(syn.OCC if kind == 0 else syn.SPIN, cells=(6, 7, 6), nsite=3, nmodels=2, seed=110 + nsb)
    q = syn.QGrid(tuple(-1.0 - 1.0 / n for n in m.cells), tuple(1.0 / n for n in m.cells),
                  tuple(n + 3 for n in m.cells))
    lm = to_library(ctx, m)
    # exact hkl = G / n (the float grid h0 + i * step misses Q = 0 by rounding)
    want = noise.subbox_intensity(m, disorder, mode, nsb, q.g_index(m.cells) / np.array(m.cells, dtype=float))
    for prec, tag in PREC:
        got, _ = lm.intensity(qgrid_tuple(q), disorder=kind, mode=mode, precision=prec, smoothing=2, subbox_n=nsb)
        assert rel_err_of_peak(got, want) < TOL[tag]


@pytest.mark.parametrize("disorder,kind,ff,mode", [("occ", 0, "const", 1), ("spin", 1, "one_j0", 0),
                                                   ("spin", 1, "const", 1)])
def test_subbox_residue_classes_against_brute_force(ctx, disorder, kind, ff, mode):
    """Sub-boxes on special positions (periods 4, 3, 2; one form-factor class): the library forms
    the pair contraction once per residue class of zones; against the oracle's literal loop over
    origins, FP64 and FP32."""
    m = _special_positions_case(kind, 6, ff, 300 + kind)
    q = m.qgrid
    lm = to_library(ctx, m)
    want = noise.subbox_intensity(m, disorder, mode, 2, q.g_index(m.cells) / np.array(m.cells, dtype=float))
    for prec, tag in PREC:
        got, _ = lm.intensity(qgrid_tuple(q), disorder=kind, mode=mode, precision=prec, smoothing=2, subbox_n=2)
        assert rel_err_of_peak(got, want) < TOL[tag]


# ----------------------------------------------------------------------------------------------
# sub-boxes by direct summation over origins (Section V A)
# ----------------------------------------------------------------------------------------------

@pytest.mark.parametrize("prec,tag", PREC)
@pytest.mark.parametrize("disorder,kind", [("occ", 0), ("spin", 1), ("disp", 2)])
@pytest.mark.parametrize("mode", [0, 1])
def test_subbox_points_random_origins(ctx, prec, tag, disorder, kind, mode):
    """Random-origin sub-boxes (the original variant of Section V A) at arbitrary Q on a
    triclinic cell with mixed form factors, 301 points (three blocks and a ragged tail), against
    the oracle's literal loop over the same origins; displacive boxes use exact exponentials."""
    m = syn.small_case(kind, cells=(6, 5, 7), nsite=3, nmodels=2, seed=150 + kind, sigma=0.1)
    lm = to_library(ctx, m)
    rng = np.random.default_rng(20 + kind)
    hkl = rng.uniform(-2.0, 2.0, (301, 3))
    org = syn.random_origins(rng, m.nmodels, m.cells, 9)
    got, info = lm.subbox_points(hkl, org, disorder=kind, mode=mode, precision=prec, subbox_n=3)
    assert info["nvox"] == hkl.shape[0]
    want = noise.subbox_intensity(m, disorder, mode, 3, hkl, org)
    assert rel_err_of_peak(got, want) < TOL[tag]


@pytest.mark.parametrize("disorder,kind", [("occ", 0), ("spin", 1)])
def test_subbox_points_every_origin_equals_pair_route(ctx, disorder, kind):
    """Every lattice point an origin, at the supercell Bragg positions: the direct sum over boxes
    equals the GPU's pair-spectrum route (DS_SMOOTH_SUBBOX on the grid) and the oracle."""
    m = syn.small_case(kind, cells=(6, 7, 6), nsite=3, nmodels=2, seed=160 + kind)
    q = syn.QGrid(tuple(-1.0 - 1.0 / n for n in m.cells), tuple(1.0 / n for n in m.cells),
                  tuple(n + 3 for n in m.cells))
    lm = to_library(ctx, m)
    hkl = q.g_index(m.cells) / np.array(m.cells, dtype=float)
    want = noise.subbox_intensity(m, disorder, 1, 2, hkl)
    for prec, tag in PREC:
        grid, _ = lm.intensity(qgrid_tuple(q), disorder=kind, mode=1, precision=prec, smoothing=2, subbox_n=2)
        pts, _ = lm.subbox_points(hkl, None, disorder=kind, mode=1, precision=prec, subbox_n=2)
        assert rel_err_of_peak(pts, grid.reshape(-1)) < TOL[tag]
        assert rel_err_of_peak(pts, want) < TOL[tag]


@pytest.mark.parametrize("prec,tag", PREC)
def test_subbox_points_displacive_every_origin_and_whole_box(ctx, prec, tag):
    """Displacive sub-boxes, every origin, against the oracle; and n_sb = n (one box spanning the
    supercell) at Bragg positions against the exact direct sum F - <F> (no Taylor expansion on
    either side), device points and device output."""
    import torch
    m = syn.small_case(syn.DISP, cells=(4, 3, 5), nsite=2, nmodels=2, seed=170, sigma=0.15)
    lm = to_library(ctx, m)
    rng = np.random.default_rng(31)
    hkl = np.concatenate([rng.uniform(-2.5, 2.5, (61, 3)), [[1.0, -1.0, 2.0], [0.0, 0.0, 0.0]]])
    for mode in (0, 1):
        got, _ = lm.subbox_points(hkl, None, disorder=2, mode=mode, precision=prec, subbox_n=2)
        assert rel_err_of_peak(got, noise.subbox_intensity(m, "disp", mode, 2, hkl)) < TOL[tag]
    hb = rng.uniform(-3.0, 3.0, (40, 3))
    org = np.array([[0, 1, 2, 3], [1, 0, 0, 0], [0, 3, 0, 1], [1, 2, 1, 4]], dtype=np.int32)
    dt = torch.float64 if prec == 0 else torch.float32
    out = torch.empty(hb.shape[0], dtype=dt, device="cuda")
    for mode in (0, 1):
        lm.subbox_points(torch.from_numpy(hb).cuda(), org, out=out, disorder=2, mode=mode, precision=prec,
                         subbox_n=3)
        torch.cuda.synchronize()
        assert rel_err_of_peak(out.cpu().numpy(), noise.subbox_intensity(m, "disp", mode, 3, hb, org)) < TOL[tag]
    whole = syn.small_case(syn.DISP, cells=(3, 3, 3), nsite=2, nmodels=2, seed=171, sigma=0.15)
    lw = to_library(ctx, whole)
    G3 = rng.integers(-7, 8, (50, 3))
    G3[0] = (3, 0, -3)
    h3 = G3 / 3.0
    org3 = np.array([[0, 1, 2, 0], [1, 2, 1, 1], [1, 0, 0, 0], [0, 0, 0, 1]], dtype=np.int32)  # two per supercell
    for mode in (0, 1):
        got, _ = lw.subbox_points(h3, org3, disorder=2, mode=mode, precision=prec, subbox_n=3)
        want = core.displacive_intensity_direct(whole, h3, mode)
        assert rel_err_of_peak(got, want) < TOL[tag]


def test_subbox_points_errors(ctx):
    import paper_1809_07088_gb300 as ds
    m = syn.small_case(syn.OCC, cells=(4, 4, 4), nsite=2, nmodels=1, seed=172)
    lm = to_library(ctx, m)
    hkl = np.zeros((3, 3))
    with pytest.raises(ds.DSError):
        lm.subbox_points(hkl, np.array([[1, 0, 0, 0]], dtype=np.int32), disorder=0, subbox_n=2)  # model 1 of 1
    with pytest.raises(ds.DSError):
        lm.subbox_points(hkl, np.array([[0, 4, 0, 0]], dtype=np.int32), disorder=0, subbox_n=2)
    with pytest.raises(ds.DSError):
        lm.subbox_points(hkl, None, disorder=0, subbox_n=0)
    with pytest.raises(ds.DSError):
        lm.subbox_points(hkl, None, disorder=0, subbox_n=5)        # n_sb > n_alpha
    with pytest.raises(ds.DSError):
        lm.subbox_points(hkl, None, disorder=1, subbox_n=2)        # no spins uploaded
    with pytest.raises(ds.DSError):
        lm.subbox_points(np.array([[np.inf, 0.0, 0.0]]), None, disorder=0, subbox_n=2)
    out, info = lm.subbox_points(np.zeros((0, 3)), None, disorder=0, subbox_n=2)
    assert out.shape == (0,) and info["nvox"] == 0


# ----------------------------------------------------------------------------------------------
# Debye-Waller factor and the magnetic + displacive coupling (Eqs. dw, mag_sf)
# ----------------------------------------------------------------------------------------------

def _mag_disp_case(seed, cells=(5, 4, 6), nsite=3):
    m = syn.small_case(syn.SPIN, cells=cells, nsite=nsite, nmodels=2, seed=seed)
    m.disp = syn.gaussian_displacements(np.random.default_rng(seed + 1), m.nmodels, m.nsite, m.cells, 0.1)
    return m


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-6)])
def test_debye_waller_points(ctx, prec, tol):
    """T_mu(Q) (Eq. dw, even part) at 257 arbitrary points, unweighted and weighted by the
    occupancies, against the oracle's direct mean (absolute error; |T| <= 1)."""
    m = syn.small_case(syn.DISP, cells=(6, 5, 4), nsite=3, nmodels=2, seed=180, sigma=0.12)
    lm = to_library(ctx, m)
    hkl = np.random.default_rng(41).uniform(-4.0, 4.0, (257, 3))
    for occw in (False, True):
        got = lm.debye_waller(hkl, precision=prec, occupancy_weights=occw)
        want = core.debye_waller(m, hkl, occupancy=occw)
        assert got.shape == want.shape
        assert np.max(np.abs(got - want)) < tol


@pytest.mark.parametrize("prec,tag", PREC)
@pytest.mark.parametrize("mode", [0, 1])
def test_magnetic_debye_waller_coupling(ctx, prec, tag, mode):
    """Eq. mag_sf with T_mu(G) of the uploaded displacements (dw_coupling = 1) on the grid of
    Bragg positions (triclinic, Q = 0 included) against the oracle's FFT method with the same
    factor; and at arbitrary points through the Lanczos route."""
    m = _mag_disp_case(190)
    lm = to_library(ctx, m)
    got, _ = lm.intensity(qgrid_tuple(m.qgrid), disorder=1, mode=mode, precision=prec, dw_coupling=1)
    want = core.magnetic_intensity_fft(m, _G(m), mode, dw=True)
    assert rel_err_of_peak(got, want) < TOL[tag]
    plain, _ = lm.intensity(qgrid_tuple(m.qgrid), disorder=1, mode=mode, precision=prec)
    assert rel_err_of_peak(plain, want) > 1e-3
    hkl = np.random.default_rng(43).uniform(-0.9, 0.9, (90, 3))
    gp, _ = lm.intensity_points(hkl, disorder=1, mode=mode, precision=prec, dw_coupling=1)
    wp = noise.lanczos_resample(lambda G: core.magnetic_intensity_fft(m, G, mode, dw=True),
                                hkl * np.array(m.cells), 2, 2)
    assert rel_err_of_peak(gp, wp) < TOL[tag]


def test_magnetic_debye_waller_errors(ctx):
    import paper_1809_07088_gb300 as ds
    m = _mag_disp_case(191, cells=(4, 4, 4), nsite=2)
    lm = to_library(ctx, m)
    q = qgrid_tuple(m.qgrid)
    with pytest.raises(ds.DSError):
        lm.intensity(q, disorder=2, dw_coupling=1)                     # not magnetic
    with pytest.raises(ds.DSError):
        lm.intensity(q, disorder=1, dw_coupling=1, smoothing=2, subbox_n=2)
    with pytest.raises(ds.DSError):
        lm.intensity(q, disorder=1, dw_coupling=2)
    with pytest.raises(ds.DSError):
        lm.backward(q, np.ones(m.qgrid.count, dtype=np.float32), disorder=1, mode=0, dw_coupling=1)
    nodisp = to_library(ctx, m, with_disp=False)
    with pytest.raises(ds.DSError):
        nodisp.intensity(q, disorder=1, dw_coupling=1)


# ----------------------------------------------------------------------------------------------
# adjoint
# ----------------------------------------------------------------------------------------------

@pytest.mark.parametrize("kern", KERNELS)
@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 2e-4)])
def test_displacive_gradient_against_oracle(ctx, prec, tol, kern):
    """dchi^2/du through ds_backward (Taylor order high enough that truncation is below
    rounding) against the oracle's chain rule of the exact direct sum, TOTAL mode."""
    from oracle import adjoint
    m = syn.small_case(syn.DISP, cells=(3, 4, 3), nsite=2, nmodels=2, seed=121, sigma=0.05)
    t = syn.small_case(syn.DISP, cells=(3, 4, 3), nsite=2, nmodels=2, seed=122, sigma=0.04)
    hkl = m.qgrid.g_index(m.cells) / np.array(m.cells, dtype=float)
    target = core.displacive_intensity_direct(t, hkl, core.TOTAL)
    chi2, g_or = adjoint.displacive_chi2_grad(m, hkl, target)
    I = core.displacive_intensity_direct(m, hkl, core.TOTAL)
    dLdI = (2.0 * (I - target)).reshape(m.qgrid.count)
    lm = to_library(ctx, m)
    dt = np.float64 if prec == 0 else np.float32
    g = lm.backward(qgrid_tuple(m.qgrid), np.ascontiguousarray(dLdI, dtype=dt), disorder=2, mode=0,
                    precision=prec, taylor_order=16, taylor_kernel=kern)
    assert g.shape == g_or.shape
    assert np.max(np.abs(g - g_or)) < tol * np.max(np.abs(g_or))


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_magnetic_gradient_against_oracle(ctx, prec, tol):
    from oracle import adjoint
    m = syn.small_case(syn.SPIN, cells=(4, 3, 5), nsite=3, nmodels=1, seed=123)
    t = syn.small_case(syn.SPIN, cells=(4, 3, 5), nsite=3, nmodels=1, seed=124)
    hkl = m.qgrid.g_index(m.cells) / np.array(m.cells, dtype=float)
    target = core.magnetic_intensity_direct(t, hkl, core.TOTAL)
    chi2, g_or = adjoint.magnetic_chi2_grad(m, hkl, target)
    I = core.magnetic_intensity_direct(m, hkl, core.TOTAL)
    dLdI = (2.0 * (I - target)).reshape(m.qgrid.count)
    lm = to_library(ctx, m)
    dt = np.float64 if prec == 0 else np.float32
    g = lm.backward(qgrid_tuple(m.qgrid), np.ascontiguousarray(dLdI, dtype=dt), disorder=1, mode=0,
                    precision=prec)
    assert np.max(np.abs(g - g_or)) < tol * np.max(np.abs(g_or))


def test_autograd_function_directional_derivative(ctx):
    """torch.autograd through the library: <grad, v> equals the central difference of the
    FP64 forward along v (dot-product test of the adjoint)."""
    import torch
    from paper_1809_07088_gb300.autograd import diffuse_intensity
    m = syn.small_case(syn.DISP, cells=(4, 4, 4), nsite=2, nmodels=1, seed=125, sigma=0.05)
    lm = to_library(ctx, m)
    q = qgrid_tuple(m.qgrid)
    u = torch.tensor(m.disp, dtype=torch.float32, device="cuda", requires_grad=True)
    I = diffuse_intensity(lm, u, q, taylor_order=14, precision=0)
    w = torch.linspace(-1.0, 1.0, I.numel(), device="cuda", dtype=I.dtype).reshape(I.shape)
    L = (I * w).sum()
    L.backward()
    gu = u.grad.double().cpu().numpy()
    rng = np.random.default_rng(0)
    v = rng.standard_normal(m.disp.shape)
    h = 1e-3
    vals = []
    for sgn in (1, -1):
        up = torch.tensor(m.disp.astype(np.float64) + sgn * h * v, dtype=torch.float32, device="cuda")
        Ip = diffuse_intensity(lm, up, q, taylor_order=14, precision=0)
        vals.append(float((Ip * w).sum()))
    fd = (vals[0] - vals[1]) / (2 * h)
    ad = float(np.sum(gu * v))
    assert abs(fd - ad) < 2e-3 * max(1.0, abs(ad))


def test_fcc_32cubed_displacive_full_size():
    """fcc 32^3 (131,072 atoms), u ~ N(0, 0.1^2), |h,k,l| <= 5 step 1/32 (321^3 voxels), Taylor
    order by the remainder bound at eps = 1e-8: FP32 within 1e-5 of peak of the FP64 path on the
    whole volume, and both within the bound of the exact direct sum on sampled voxels."""
    import torch
    m, _ = syn.differentiation_pair()
    lm = to_library(ctx_holder(), m)
    q = qgrid_tuple(m.qgrid)
    o32 = torch.empty(m.qgrid.count, dtype=torch.float32, device="cuda")
    o64 = torch.empty(m.qgrid.count, dtype=torch.float64, device="cuda")
    _, info = lm.intensity(q, out=o32, disorder=2, mode=0, precision=1, taylor_order=-1, taylor_eps=1e-8)
    lm.intensity(q, out=o64, disorder=2, mode=0, precision=0, taylor_order=-1, taylor_eps=1e-8)
    torch.cuda.synchronize()
    peak = float(o64.max())
    assert float((o32.double() - o64).abs().max()) < 1e-5 * peak
    P = info["taylor_order"]
    assert P == core.taylor_order(core.x_max(m, m.qgrid), 1e-8)
    idx = np.random.default_rng(7).choice(m.qgrid.nvox, 200, replace=False)
    hkl = sample_G(m, idx) / 32.0
    I_dir, F = core.displacive_intensity_direct(m, hkl, 0, return_F=True)
    bound = core.truncation_bound(m, hkl, P, 0, F=F)
    sel = torch.from_numpy(idx).cuda()
    for out, tol in ((o64, 1e-10), (o32, 1e-5)):
        got = out.reshape(-1)[sel].double().cpu().numpy()
        assert np.all(np.abs(got - I_dir) <= bound + tol * peak)


def test_fcc_32cubed_gradient_directional_derivative():
    """Full-size adjoint: chi^2 against the correlated target model; <dchi2/du, v> from the
    FP32 adjoint against the central difference of the FP64 forward along a random v."""
    import torch
    m, t = syn.differentiation_pair()
    ctx = ctx_holder()
    lm, lt = to_library(ctx, m), to_library(ctx, t)
    q = qgrid_tuple(m.qgrid)
    opts = dict(disorder=2, mode=0, taylor_order=-1, taylor_eps=1e-8)
    It = torch.empty(m.qgrid.count, dtype=torch.float64, device="cuda")
    lt.intensity(q, out=It, precision=0, **opts)
    I = torch.empty(m.qgrid.count, dtype=torch.float64, device="cuda")
    lm.intensity(q, out=I, precision=0, **opts)
    dL = (2.0 * (I - It)).float().contiguous()
    g = torch.empty(lm._shape(3), dtype=torch.float32, device="cuda")
    lm.backward(q, dL, grad=g, precision=1, **opts)
    v = torch.from_numpy(np.random.default_rng(3).standard_normal(m.disp.shape)).cuda()
    h = 2e-4
    chi = []
    for sgn in (1, -1):
        lm.upload_displacements(torch.from_numpy(m.disp.astype(np.float64)).cuda().add(sgn * h * v).float().contiguous())
        lm.intensity(q, out=I, precision=0, **opts)
        chi.append(float(((I - It) ** 2).sum()))
    fd = (chi[0] - chi[1]) / (2 * h)
    ad = float((g.double() * v).sum())
    assert abs(fd - ad) < 2e-3 * abs(ad)


def test_perovskite_64cubed_displacive_full_size():
    """Perovskite 64^3 (1,310,720 atoms), correlated displacements, 4-Gaussian form factors,
    |h,k,l| <= 8 step 1/64 (1025^3 voxels), FP32 with eps = 1e-5: sampled voxels against the
    exact direct sum within the remainder bound + 1e-5 of peak; the Lanczos (m = 2, m' = 8)
    volume at sampled voxels against the literal finite sum over direct-sum I(G)."""
    import torch
    m = syn.perovskite_correlated()
    lm = to_library(ctx_holder(), m)
    q = qgrid_tuple(m.qgrid)
    out = torch.empty(m.qgrid.count, dtype=torch.float32, device="cuda")
    _, info = lm.intensity(q, out=out, disorder=2, mode=1, precision=1, taylor_order=-1, taylor_eps=1e-5)
    torch.cuda.synchronize()
    peak = float(out.max())
    P = info["taylor_order"]
    # the order chosen by the library is the oracle's: the smallest order whose remainder bound
    # x_max^(P+1)/(P+1)! <= eps, x_max over the atoms and the corners of the whole grid
    assert P == core.taylor_order(core.x_max(m, m.qgrid), 1e-5)
    idx = np.random.default_rng(11).choice(m.qgrid.nvox, 40, replace=False)
    hkl = sample_G(m, idx) / 64.0
    I_dir, F = core.displacive_intensity_direct(m, hkl, 1, return_F=True)
    bound = core.truncation_bound(m, hkl, P, 1, F=F)
    got = out.reshape(-1)[torch.from_numpy(idx).cuda()].double().cpu().numpy()
    assert np.all(np.abs(got - I_dir) <= bound + 1e-5 * peak)
    del out
    torch.cuda.empty_cache()
    sm = torch.empty(m.qgrid.count, dtype=torch.float32, device="cuda")
    lm.intensity(q, out=sm, disorder=2, mode=1, precision=1, taylor_order=P, smoothing=1, lanczos_m=2,
                 lanczos_mprime=8)
    torch.cuda.synchronize()
    pick = np.array([[512, 512, 512], [300, 700, 650], [64, 900, 512]])
    Q = pick + sample_G(m, np.array([0]))[0]
    IG = lambda Gs: core.displacive_intensity_direct(m, Gs / 64.0, 1)
    want = noise.lanczos_resample(IG, Q.astype(np.float64), 2, 8)
    got = np.array([float(sm[tuple(p)]) for p in pick])
    assert np.all(np.abs(got - want) <= 1e-5 * float(sm.max()) + 1e-4 * np.abs(want))


def test_perovskite_64cubed_fp32_against_fp64_on_corner_and_centre_zones():
    """The perovskite 64^3 model (1,310,720 atoms, x_max ~ 8.6 on |h,k,l| <= 8, where the
    alternating Taylor terms cancel most) at the oracle's order for eps = 1e-5 over the whole
    grid: on every voxel of the two |Q|-maximal corner zones H = (7, 7, 7) (voxels up to
    h = 7 + 63/64) and H = (-8, -8, -8) (down to h = -8), and of the centre zone H = (0, 0, 0),
    the FP32 path is within 1e-5 of peak of the FP64 path with the same P; 420 voxels of those
    zones (the Bragg position and the outermost corner of each included) are within the per-voxel
    remainder bound of Section III C (+ 1e-5 of peak) of the exact direct sum, on both paths."""
    import torch
    m = syn.perovskite_correlated()
    lm = to_library(ctx_holder(), m)
    P = core.taylor_order(core.x_max(m, m.qgrid), 1e-5)
    assert P >= 25
    zones = [(7, 7, 7), (-8, -8, -8), (0, 0, 0)]
    n = m.cells[0]
    got = {}
    for H in zones:
        q = (tuple(float(h) for h in H), (1.0 / n,) * 3, (n, n, n))
        for prec, dt in ((0, torch.float64), (1, torch.float32)):
            o = torch.empty((n, n, n), dtype=dt, device="cuda")
            _, info = lm.intensity(q, out=o, disorder=2, mode=1, precision=prec, taylor_order=P,
                                   taylor_kernel=1)
            assert info["taylor_order"] == P
            got[H, prec] = o
        torch.cuda.synchronize()
    peak = max(float(got[H, 0].max()) for H in zones)
    for H in zones:
        err = float((got[H, 1].double() - got[H, 0]).abs().max()) / peak
        assert err < 1e-5, (H, err)
    # the sum-factorised kernel forced on the outermost zone (FP32) against the per-voxel FP64 path
    q = ((7.0, 7.0, 7.0), (1.0 / n,) * 3, (n, n, n))
    o = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    lm.intensity(q, out=o, disorder=2, mode=1, precision=1, taylor_order=P, taylor_kernel=2)
    torch.cuda.synchronize()
    assert float((o.double() - got[(7, 7, 7), 0]).abs().max()) / peak < 1e-5
    rng = np.random.default_rng(21)
    G, vals = [], {0: [], 1: []}
    for H in zones:
        ijk = np.concatenate([rng.integers(0, n, (138, 3)), [[0, 0, 0], [n - 1, n - 1, n - 1]]])
        G.append(np.asarray(H)[None, :] * n + ijk)
        sel = torch.from_numpy(np.ravel_multi_index(ijk.T, (n, n, n))).cuda()
        for prec in (0, 1):
            vals[prec].append(got[H, prec].reshape(-1)[sel].double().cpu().numpy())
    hkl = np.concatenate(G) / float(n)
    I_dir, F = core.displacive_intensity_direct(m, hkl, 1, return_F=True)
    bound = core.truncation_bound(m, hkl, P, 1, F=F, chunk=32)
    for prec in (0, 1):
        v = np.concatenate(vals[prec])
        assert np.all(np.abs(v - I_dir) <= bound + 1e-5 * peak), prec


def test_subbox_random_displacive_fcc32_plane_full_size():
    """The sub-box row at full size: fcc 32^3, u ~ N(0, 0.1^2), n_sb = 5, random origins covering
    every lattice point, (h h l) plane 201 x 201 on the device, DIFFUSE, FP32: sampled points
    (one on a Bragg position) against the oracle's loop over the same origins; the FP64 path on
    the same points within 1e-10."""
    import torch
    m = syn.displacive_fcc(cells=(32, 32, 32), sigma=0.1, seed=5)
    lm = to_library(ctx_holder(), m)
    org = syn.covering_origins(np.random.default_rng(7), 1, m.cells, 5)
    u, v = np.meshgrid(np.linspace(-5.0, 5.0, 201), np.linspace(-5.0, 5.0, 201), indexing="ij")
    hkl = np.stack([u.ravel(), u.ravel(), v.ravel()], axis=1)
    out = torch.empty(hkl.shape[0], dtype=torch.float32, device="cuda")
    lm.subbox_points(torch.from_numpy(hkl).cuda(), org, out=out, disorder=2, mode=1, precision=1, subbox_n=5)
    torch.cuda.synchronize()
    pick = np.concatenate([np.random.default_rng(11).choice(hkl.shape[0], 7, replace=False), [100 * 201 + 100]])
    want = noise.subbox_intensity(m, "disp", 1, 5, hkl[pick], org)
    peak = float(out.max())
    assert np.max(np.abs(out.cpu().numpy()[pick] - want)) < 1e-5 * peak
    g64, _ = lm.subbox_points(hkl[pick], org, disorder=2, mode=1, precision=0, subbox_n=5)
    assert rel_err_of_peak(g64, want) < TOL["fp64"]


def test_magnetic_debye_waller_pyrochlore20_full_size():
    """The Debye-Waller coupling row at full size: magnetic pyrochlore 20^3 with u ~ N(0, 0.05^2),
    |h,k,l| <= 2 step 1/20 (81^3 voxels), FP32 on the device: sampled voxels (Q = 0 included)
    against the oracle's direct sum with T_mu(G)."""
    import torch
    m = syn.pyrochlore_mag_disp(cells=(20, 20, 20), hmax=2.0)
    lm = to_library(ctx_holder(), m)
    out = torch.empty(m.qgrid.count, dtype=torch.float32, device="cuda")
    lm.intensity(qgrid_tuple(m.qgrid), out=out, disorder=1, mode=0, precision=1, dw_coupling=1)
    torch.cuda.synchronize()
    idx = np.concatenate([np.random.default_rng(12).choice(m.qgrid.nvox, 300, replace=False),
                          [np.ravel_multi_index((40, 40, 40), m.qgrid.count)]])
    hkl = sample_G(m, idx) / 20.0
    want = core.magnetic_intensity_direct(m, hkl, 0, dw=True)
    got = out.reshape(-1)[torch.from_numpy(idx).cuda()].double().cpu().numpy()
    assert np.max(np.abs(got - want)) < 1e-5 * float(out.max())


_CTX = []


def sample_G(m, idx):
    """Supercell indices G of the voxels `idx` of m.qgrid without building the whole grid."""
    g0 = np.rint(np.array(m.qgrid.h0) * np.array(m.cells)).astype(np.int64)
    ijk = np.stack(np.unravel_index(np.asarray(idx), m.qgrid.count), axis=1)
    return g0[None, :] + ijk


def ctx_holder():
    import paper_1809_07088_gb300 as ds
    if not _CTX:
        _CTX.append(ds.Context(0))
    return _CTX[0]
