"""Listmode PET on the GPU against the FP64 oracle, through the C ABI.

The system matrix of Sec. 2.1.1, Eq. (2) (Joseph line integrals, Gaussian
resolution model, attenuation and normalisation factors) and listmode OSEM
(Table 1).  Bars: projections, attenuation factors and back projections
within relative L2 1e-5 of FP64; OSEM images within 2e-5; the listmode
count identity sum (sens / M) x_new = sum p / (p + s) in FP64 diagnostics;
at the full 204 x 204 x 154 grid, sampled lines match the oracle one by one
and the count identity holds for a whole subiteration.

The oracle decides Joseph's integers (principal axis, planes, time-of-flight
window) in double precision, the kernel the axis and planes in single
precision: the few lines where the two differ (rounding ties) are left out
of each comparison and counted (pet_precision.py).
"""
import dataclasses

import numpy as np
import pytest

from helpers import rel_l2
from pet_precision import keep_alike

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pet_mods(spect_lib, oracle_mod):
    from oracle import pet as opet
    from paper_2309_01977_gb300 import pet, pet_phantom
    return pet, pet_phantom, opet


@pytest.fixture(scope="module")
def small(pet_mods):
    pet, pp, opet = pet_mods
    wl = pp.PET_WORKLOADS["petlm_small"]
    act, mu, semi = pp.head_phantom(wl.shape, wl.voxel, wl.seed)
    lors, eta, s, _, _ = pp.draw_events(wl, act, semi)
    og = opet.PetGeom(wl.shape, wl.voxel, rr_sigma_mm=np.float32(wl.rr_sigma_mm), rr_nsigma=3.0)
    return wl, act.numpy(), mu.numpy(), lors.numpy(), eta.numpy(), s.numpy(), og


def _odd_lors(wl, seed, count=600):
    """Lines with ends inside the image, axis-parallel lines, steep lines,
    degenerate (zero-length) lines and lines that miss the image."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ext = 0.5 * np.asarray(wl.shape) * np.asarray(wl.voxel)
    out = []
    for i in range(count):
        k = i % 5
        if k == 0:
            p = rng.uniform(-ext, ext, size=(2, 3)).ravel()
        elif k == 1:
            ax = rng.integers(3)
            c = rng.uniform(-ext, ext)
            a, b = c.copy(), c.copy()
            a[ax], b[ax] = -3 * ext[ax], 3 * ext[ax]
            p = np.concatenate([a, b])
        elif k == 2:
            c = rng.uniform(-0.5 * ext, 0.5 * ext)
            d = np.array([rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), 1.0])
            p = np.concatenate([c - 400 * d, c + 400 * d])
        elif k == 3:
            c = rng.uniform(-ext, ext)
            p = np.concatenate([c, c])
        else:
            p = np.concatenate([[-500.0, 3 * ext[1], 0.0], [500.0, 3 * ext[1] + 10.0, 5.0]])
        out.append(p)
    return np.asarray(out, dtype=np.float32)


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).to(dev)


def _plan(pet, wl, mu, dev, rr=True, subsets=None):
    g = pet.PetGeometry(wl.shape, wl.voxel, rr_sigma_mm=wl.rr_sigma_mm if rr else 0.0,
                        n_subsets=subsets or wl.n_subsets, n_tof_bins=wl.tof_bins, tof_bin_mm=wl.tof_bin_mm,
                        tof_sigma_mm=wl.tof_sigma_mm)
    return pet.PetPlan(g, None if mu is None else _t(mu, dev), stream=torch.cuda.current_stream())


def test_forward_matches_oracle(pet_mods, small, cuda):
    pet, pp, opet = pet_mods
    wl, act, mu, lors, eta, s, og = small
    L = np.concatenate([lors[:6000], _odd_lors(wl, 5)])
    L = L[keep_alike(L, og, opet)]
    rng = np.random.Generator(np.random.PCG64(6))
    x = (act + rng.uniform(0, 0.5, size=act.shape)).astype(np.float32)
    m = rng.uniform(0.5, 1.0, size=len(L)).astype(np.float32)
    plan = _plan(pet, wl, mu, cuda)
    got = plan.forward(_t(x, cuda), _t(L, cuda), _t(m, cuda)).cpu().numpy()
    ref = opet.forward(x, L, og, m)
    err = rel_l2(got, ref)
    print("PET forward (T_rr + Joseph) rel L2 vs FP64: %.2e" % err)
    assert err <= 1e-5
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))
    # degenerate and missing lines are exactly 0 on both sides
    zero = ref == 0.0
    assert np.all(got[zero] == 0.0)
    plan.close()


def test_forward_without_resolution_model(pet_mods, small, cuda):
    pet, pp, opet = pet_mods
    wl, act, mu, lors, eta, s, og = small
    L = np.concatenate([lors[:3000], _odd_lors(wl, 7)])
    L = L[keep_alike(L, og, opet)]
    plan = _plan(pet, wl, None, cuda, rr=False)
    got = plan.forward(_t(act, cuda), _t(L, cuda)).cpu().numpy()
    ref = opet.joseph_fwd(act, L, dataclasses.replace(og, rr_sigma_mm=0.0))
    assert rel_l2(got, ref) <= 1e-5
    plan.close()


def test_mult_matches_oracle(pet_mods, small, cuda):
    pet, pp, opet = pet_mods
    wl, act, mu, lors, eta, s, og = small
    L = np.concatenate([lors[:5000], _odd_lors(wl, 8)])
    e = np.concatenate([eta[:5000], np.full(len(L) - 5000, 0.9, dtype=np.float32)])
    keep = keep_alike(L, og, opet)
    L, e = L[keep], e[keep]
    plan = _plan(pet, wl, mu, cuda)
    got = plan.mult(_t(L, cuda), _t(e, cuda)).cpu().numpy()
    ref = opet.mult(L, og, mu=mu, eta=e)
    # exp(-L) carries the absolute FP32 error of the line integral L of mu
    # (a few hundred samples, L up to ~2): the FP32 bound of 1e-5
    worst = float(np.max(np.abs(got - ref) / ref))
    print("attenuation and normalisation factors: worst relative error %.2e" % worst)
    assert worst <= 1e-5
    plan.close()
    plan = _plan(pet, wl, None, cuda)
    assert np.array_equal(plan.mult(_t(L, cuda)).cpu().numpy(), np.ones(len(L), dtype=np.float32))
    plan.close()


def test_back_matches_oracle_and_is_adjoint(pet_mods, small, cuda):
    pet, pp, opet = pet_mods
    wl, act, mu, lors, eta, s, og = small
    L = np.concatenate([lors[:8000], _odd_lors(wl, 9)])
    L = L[keep_alike(L, og, opet)]
    rng = np.random.Generator(np.random.PCG64(10))
    q = rng.uniform(0.0, 2.0, size=len(L)).astype(np.float32)
    m = rng.uniform(0.5, 1.0, size=len(L)).astype(np.float32)
    plan = _plan(pet, wl, mu, cuda)
    got = plan.back(_t(q, cuda), _t(L, cuda), _t(m, cuda)).cpu().numpy()
    ref = opet.back(q, L, og, m)
    err = rel_l2(got, ref)
    print("PET back (Joseph^T + T_rr) rel L2 vs FP64: %.2e" % err)
    assert err <= 1e-5
    x = rng.uniform(size=wl.shape).astype(np.float32)
    hx = plan.forward(_t(x, cuda), _t(L, cuda), _t(m, cuda)).double().cpu().numpy()
    lhs = float(np.dot(hx, q))
    rhs = float(np.sum(x.astype(np.float64) * got))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    plan.close()


def test_empty_lists(pet_mods, small, cuda):
    pet, pp, opet = pet_mods
    wl, act, mu, lors, eta, s, og = small
    plan = _plan(pet, wl, mu, cuda)
    L = torch.zeros((0, 6), device=cuda)
    assert plan.forward(_t(act, cuda), L).numel() == 0
    b = plan.back(torch.zeros(0, device=cuda), L)
    assert float(b.abs().sum()) == 0.0
    plan.close()


def _osem_inputs(pet, pp, opet, wl, mu, lors, eta, og):
    L_all, eta_all, w = pp.scanner_lors(wl.scanner, eff_seed=wl.seed)
    m_all = opet.mult(L_all.numpy(), og, mu=mu, eta=eta_all.numpy())
    sens = (w * opet.back(np.ones(len(m_all)), L_all.numpy(), og, m_all)).astype(np.float32)
    mult = opet.mult(lors, og, mu=mu, eta=eta).astype(np.float32)
    return sens, mult


def test_lm_osem_matches_oracle(pet_mods, small, cuda):
    pet, pp, opet = pet_mods
    wl, act, mu, lors, eta, s, og = small
    keep = keep_alike(lors, og, opet)
    lors, eta, s = lors[keep], eta[keep], s[keep]
    sens, mult = _osem_inputs(pet, pp, opet, wl, mu, lors, eta, og)
    M, n_sub = wl.n_subsets, wl.n_subsets * wl.n_iters
    ref, rdiag = opet.lm_osem(lors, mult, s, sens, og, M, count=n_sub)
    plan = _plan(pet, wl, mu, cuda)
    x = torch.ones(wl.shape, device=cuda)
    diag = plan.lm_osem(_t(lors, cuda), _t(mult, cuda), _t(s, cuda), _t(sens, cuda), x, 0, n_sub, diag=True)
    err = rel_l2(x.cpu().numpy(), ref)
    print("PET listmode OSEM %dx%d image rel L2 vs FP64: %.2e" % (wl.n_iters, M, err))
    assert err <= 2e-5
    for k in range(n_sub):
        assert diag[k][1] == rdiag[k][1]
        assert abs(diag[k][0] - rdiag[k][0]) <= 2e-5 * rdiag[k][0]
    plan.close()


def test_lm_osem_count_identity(pet_mods, small, cuda):
    pet, pp, opet = pet_mods
    wl, act, mu, lors, eta, s, og = small
    sens, mult = _osem_inputs(pet, pp, opet, wl, mu, lors, eta, og)
    M = wl.n_subsets
    plan = _plan(pet, wl, mu, cuda)
    x = torch.ones(wl.shape, device=cuda)
    sens_t = _t(sens, cuda)
    for it in range(2 * M):
        for s_arr in (None, _t(s, cuda)):
            xx = x.clone()
            d = plan.lm_osem(_t(lors, cuda), _t(mult, cuda), s_arr, sens_t, xx, it, 1, diag=True)[0]
            lhs = float((sens_t.double() / M * xx.double()).sum())
            assert abs(lhs - d[0]) <= 2e-5 * d[0]
            if s_arr is None:  # every counted event contributes p / p = 1
                assert d[0] == d[1] <= len(range(it % M, len(lors), M))
        plan.lm_osem(_t(lors, cuda), _t(mult, cuda), _t(s, cuda), sens_t, x, it, 1)
    plan.close()


def test_full_grid_sampled_lines_and_count_identity(pet_mods, cuda):
    """The 204 x 204 x 154 grid and scanner of the benchmark, 3 M prompts (so
    the projection kernels run with the same grid-stride launch as at 30 M):
    2000 sampled lines match the oracle one by one; one listmode
    subiteration satisfies the count identity."""
    pet, pp, opet = pet_mods
    wl = dataclasses.replace(pp.PET_WORKLOADS["petlm204"], prompts=3_000_000)
    act, mu, semi = pp.head_phantom(wl.shape, wl.voxel, wl.seed, device=cuda)
    lors, eta, s, _, _ = pp.draw_events(wl, act, semi, device=cuda)
    plan = _plan(pet, wl, mu.cpu().numpy(), cuda)
    mult = plan.mult(lors, eta)
    p = plan.forward(act, lors, mult)
    rng = np.random.Generator(np.random.PCG64(12))
    pick = np.sort(rng.choice(lors.shape[0], 2000, replace=False))
    og = opet.PetGeom(wl.shape, wl.voxel, rr_sigma_mm=np.float32(wl.rr_sigma_mm), rr_nsigma=3.0)
    pick = pick[keep_alike(lors.cpu().numpy()[pick], og, opet)]
    L = lors.cpu().numpy()[pick]
    m_ref = opet.mult(L, og, mu=mu.cpu().numpy(), eta=eta.cpu().numpy()[pick])
    assert np.max(np.abs(mult.cpu().numpy()[pick] - m_ref) / m_ref) <= 1e-5
    ref = opet.forward(act.cpu().numpy(), L, og, mult.cpu().numpy()[pick])
    got = p.cpu().numpy()[pick]
    err = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)))
    print("PET 204^3-grid sampled lines: max rel err %.2e" % float(err.max()))
    assert float(err.max()) <= 1e-5
    # count identity for one subiteration at full size (sens from a quarter
    # of the crystals; any positive sens image satisfies the identity)
    L_all, eta_all, w = pp.scanner_lors(wl.scanner, angle_step=8, ring_step=4, device=cuda, eff_seed=wl.seed)
    m_all = plan.mult(L_all, eta_all)
    sens = plan.back(m_all * w, L_all)
    x = torch.ones(wl.shape, device=cuda)
    d = plan.lm_osem(lors, mult, s, sens, x, 0, 1, diag=True)[0]
    lhs = float((sens.double() / wl.n_subsets * x.double())[sens > 0].sum())
    assert abs(lhs - d[0]) <= 1e-4 * d[0]
    plan.close()


# ---------------------------------------------------------------- time of flight

@pytest.fixture(scope="module")
def small_tof(pet_mods):
    """The small case with time of flight: 15 bins over 240 mm, 250 ps."""
    pet, pp, opet = pet_mods
    wl = dataclasses.replace(pp.PET_WORKLOADS["petlm_small"], tof_bins=15, tof_range_mm=240.0, tof_fwhm_ps=250.0)
    act, mu, semi = pp.head_phantom(wl.shape, wl.voxel, wl.seed)
    lors, eta, s, _, tb = pp.draw_events(wl, act, semi)
    og = opet.PetGeom(wl.shape, wl.voxel, rr_sigma_mm=np.float32(wl.rr_sigma_mm), rr_nsigma=3.0)
    return wl, act.numpy(), mu.numpy(), lors.numpy(), eta.numpy(), s.numpy(), tb.numpy(), og


def _otof(opet, wl, bins):
    # the library holds the model in single precision; the oracle gets the same values
    return opet.Tof(n_bins=wl.tof_bins, bin_mm=float(np.float32(wl.tof_bin_mm)),
                    sigma_mm=float(np.float32(wl.tof_sigma_mm)), bins=bins, nsigma=3.0)


def _tof_model(wl, bins):
    return (wl.tof_bins, wl.tof_bin_mm, wl.tof_sigma_mm, 3.0, bins)


def _ti(a, dev):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.int32))).to(dev)


def test_tof_forward_and_back_match_oracle(pet_mods, small_tof, cuda):
    pet, pp, opet = pet_mods
    wl, act, mu, lors, eta, s, tb, og = small_tof
    L, B = lors[:8000], tb[:8000]
    keep = keep_alike(L, og, opet, _tof_model(wl, B))
    L, B = L[keep], B[keep]
    rng = np.random.Generator(np.random.PCG64(30))
    x = (act + rng.uniform(0, 0.5, size=act.shape)).astype(np.float32)
    m = rng.uniform(0.5, 1.0, size=len(L)).astype(np.float32)
    plan = _plan(pet, wl, mu, cuda)
    got = plan.forward(_t(x, cuda), _t(L, cuda), _t(m, cuda), tof_bin=_ti(B, cuda)).cpu().numpy()
    ref = opet.forward(x, L, og, m, tof=_otof(opet, wl, B))
    err = rel_l2(got, ref)
    print("PET TOF forward rel L2 vs FP64: %.2e" % err)
    assert err <= 1e-5
    q = rng.uniform(0.0, 2.0, size=len(L)).astype(np.float32)
    gb = plan.back(_t(q, cuda), _t(L, cuda), _t(m, cuda), tof_bin=_ti(B, cuda)).cpu().numpy()
    rb = opet.back(q, L, og, m, tof=_otof(opet, wl, B))
    errb = rel_l2(gb, rb)
    print("PET TOF back rel L2 vs FP64: %.2e" % errb)
    assert errb <= 1e-5
    lhs = float(np.dot(got.astype(np.float64), q))
    rhs = float(np.sum(x.astype(np.float64) * gb))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    plan.close()


def test_tof_lm_osem_matches_oracle(pet_mods, small_tof, cuda):
    pet, pp, opet = pet_mods
    wl, act, mu, lors, eta, s, tb, og = small_tof
    keep = keep_alike(lors, og, opet, _tof_model(wl, tb))
    lors, eta, s, tb = lors[keep], eta[keep], s[keep], tb[keep]
    sens, mult = _osem_inputs(pet, pp, opet, wl, mu, lors, eta, og)
    M, n_sub = wl.n_subsets, wl.n_subsets * wl.n_iters
    ref, rdiag = opet.lm_osem(lors, mult, s, sens, og, M, count=n_sub, tof=_otof(opet, wl, tb))
    plan = _plan(pet, wl, mu, cuda)
    x = torch.ones(wl.shape, device=cuda)
    diag = plan.lm_osem(_t(lors, cuda), _t(mult, cuda), _t(s, cuda), _t(sens, cuda), x, 0, n_sub, diag=True,
                        tof_bin=_ti(tb, cuda))
    err = rel_l2(x.cpu().numpy(), ref)
    print("PET TOF listmode OSEM %dx%d image rel L2 vs FP64: %.2e" % (wl.n_iters, M, err))
    assert err <= 2e-5
    for k in range(n_sub):
        assert diag[k][1] == rdiag[k][1]
        assert abs(diag[k][0] - rdiag[k][0]) <= 2e-5 * rdiag[k][0]
    plan.close()


def test_tof_full_grid_sampled_lines(pet_mods, cuda):
    """The paper's TOF model (550 ps, 21 bins over 30 cm) on the 204^3 grid,
    3 M prompts: 2000 sampled lines match the oracle one by one."""
    pet, pp, opet = pet_mods
    wl = dataclasses.replace(pp.PET_WORKLOADS["petlm204tof"], prompts=3_000_000)
    act, mu, semi = pp.head_phantom(wl.shape, wl.voxel, wl.seed, device=cuda)
    lors, eta, s, _, tb = pp.draw_events(wl, act, semi, device=cuda)
    plan = _plan(pet, wl, mu.cpu().numpy(), cuda)
    mult = plan.mult(lors, eta)
    p = plan.forward(act, lors, mult, tof_bin=tb)
    rng = np.random.Generator(np.random.PCG64(31))
    pick = np.sort(rng.choice(lors.shape[0], 2000, replace=False))
    og = opet.PetGeom(wl.shape, wl.voxel, rr_sigma_mm=np.float32(wl.rr_sigma_mm), rr_nsigma=3.0)
    pick = pick[keep_alike(lors.cpu().numpy()[pick], og, opet, _tof_model(wl, tb.cpu().numpy()[pick]))]
    ref = opet.forward(act.cpu().numpy(), lors.cpu().numpy()[pick], og, mult.cpu().numpy()[pick],
                       tof=_otof(opet, wl, tb.cpu().numpy()[pick]))
    got = p.cpu().numpy()[pick]
    err = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)))
    print("PET TOF 204^3-grid sampled lines: max rel err %.2e" % float(err.max()))
    assert float(err.max()) <= 1e-5
    plan.close()


def test_tof_bins_outside_the_range_and_bad_arguments(pet_mods, small_tof, cuda):
    """Bins past either end of the range move the window off the line (the
    projection is the Gaussian's far tail or zero on both sides); a bin array
    for a plan without time of flight and misaligned lines are rejected."""
    pet, pp, opet = pet_mods
    wl, act, mu, lors, eta, s, tb, og = small_tof
    L = lors[:400]
    B = np.where(np.arange(400) % 2 == 0, -3, wl.tof_bins + 2).astype(np.int32)
    keep = keep_alike(L, og, opet, _tof_model(wl, B))
    L, B = L[keep], B[keep]
    plan = _plan(pet, wl, mu, cuda)
    got = plan.forward(_t(act, cuda), _t(L, cuda), tof_bin=_ti(B, cuda)).cpu().numpy()
    ref = opet.forward(act, L, og, tof=_otof(opet, wl, B))
    assert np.max(np.abs(got - ref)) <= 1e-5 * max(1.0, float(np.max(np.abs(opet.forward(act, L, og)))))
    plan.close()
    no_tof = pet.PetPlan(pet.PetGeometry(wl.shape, wl.voxel), None, stream=torch.cuda.current_stream())
    with pytest.raises(pet.SpectError) as e:
        no_tof.forward(_t(act, cuda), _t(L, cuda), tof_bin=_ti(B, cuda))
    assert e.value.status == pet.SPECT_EINVAL
    lib = pet.load()
    Ld = _t(L, cuda)
    out = torch.empty(len(L) - 1, device=cuda)
    bad = Ld.data_ptr() + 4  # 4-byte offset: not 8-byte aligned
    rc = lib.pet_forward(no_tof.handle, _t(act, cuda).data_ptr(), bad, None, None, len(L) - 1, out.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    assert rc == pet.SPECT_EINVAL
    no_tof.close()
