"""CPU checks of the seeded listmode PET inputs (scanner, head phantom,
Monte Carlo events): shapes and ranges, determinism under a seed, events on
the crystal cylinder, time-of-flight bins that follow the emission point,
and the sensitivity LOR set."""
import dataclasses
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2309_01977_gb300 import pet_phantom as pp  # noqa: E402


def _small(**kw):
    return dataclasses.replace(pp.PET_WORKLOADS["petlm_small"], **kw)


def test_head_phantom_ranges():
    wl = _small()
    act, mu, semi = pp.head_phantom(wl.shape, wl.voxel, wl.seed)
    assert act.shape == mu.shape == tuple(wl.shape)
    assert float(act.min()) == 0.0 and float(act.max()) == 8.0
    vals = np.unique(mu.numpy()).astype(np.float64)
    allowed = np.array([0.0, pp.WATER_MU_MM, pp.BONE_MU_MM])
    assert all(np.min(np.abs(allowed - v)) <= 1e-8 for v in vals)
    assert all(s > 0 for s in semi)


def test_events_deterministic_and_on_the_scanner():
    wl = _small(prompts=3000)
    act, mu, semi = pp.head_phantom(wl.shape, wl.voxel, wl.seed)
    a = pp.draw_events(wl, act, semi)
    b = pp.draw_events(wl, act, semi)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    lors, eta, s, n_true, tof = a
    assert lors.shape == (3000, 6) and lors.dtype == torch.float32 and tof is None
    assert n_true == 2700
    r1 = torch.linalg.norm(lors[:, :2].double(), dim=1)
    r2 = torch.linalg.norm(lors[:, 3:5].double(), dim=1)
    assert torch.allclose(r1, torch.full_like(r1, wl.scanner.radius_mm), rtol=1e-6)
    assert torch.allclose(r2, torch.full_like(r2, wl.scanner.radius_mm), rtol=1e-6)
    assert float(lors[:, 2].abs().max()) <= wl.scanner.axial_half_mm
    assert float(eta.min()) >= 0.85 ** 2 - 1e-6 and float(eta.max()) <= 1.15 ** 2 + 1e-6
    pairs = wl.scanner.n_crystals * (wl.scanner.n_crystals - 1) / 2
    assert abs(float(s[0]) - 300 / pairs) <= 1e-6 * 300 / pairs


def test_tof_bins_follow_the_emission_point():
    """With a timing resolution far finer than a bin, a true event's bin is
    the bin of its emission point's arc length from the line's midpoint."""
    wl = _small(prompts=4000, randoms_frac=0.0, tof_bins=41, tof_range_mm=246.0, tof_fwhm_ps=1e-3)
    act, mu, semi = pp.head_phantom(wl.shape, wl.voxel, wl.seed)
    lors, eta, s, n_true, tof = pp.draw_events(wl, act, semi)
    assert tof.dtype == torch.int32 and int(tof.min()) >= 0 and int(tof.max()) < wl.tof_bins
    assert math.isclose(wl.tof_bin_mm, 6.0)
    # the bin centre, placed on the line, lies in the head ellipsoid (up to
    # half a bin): the emission point it came from is inside the head
    p1, p2 = lors[:, :3].double(), lors[:, 3:].double()
    u = (p2 - p1) / torch.linalg.norm(p2 - p1, dim=1, keepdim=True)
    c = (tof.double() - 0.5 * (wl.tof_bins - 1)) * wl.tof_bin_mm
    pt = 0.5 * (p1 + p2) + c[:, None] * u
    half = 0.5 * wl.tof_bin_mm
    grown = torch.tensor([a + half for a in semi], dtype=torch.float64)
    r = torch.sqrt(((pt / grown) ** 2).sum(dim=1))
    assert float(r.max()) <= 1.0 + 1e-9
    assert len(torch.unique(tof)) > 5


def test_sensitivity_lor_set():
    sc = pp.Scanner(radius_mm=100.0, crystals_per_ring=16, rings=4, ring_pitch_mm=5.0)
    lors, eta, w = pp.scanner_lors(sc, angle_step=2, ring_step=2, eff_seed=1)
    m = (16 // 2) * (4 // 2)
    assert lors.shape == (m * (m - 1) // 2, 6) and w == 16.0
    assert eta is not None and eta.shape[0] == lors.shape[0]
    lors1, _, w1 = pp.scanner_lors(sc)
    assert lors1.shape[0] == 64 * 63 // 2 and w1 == 1.0
