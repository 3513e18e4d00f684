"""Seeded synthetic listmode PET data: scanner, phantom and events.

Input generation only (no projector arithmetic): a cylindrical scanner of
crystal rings, a head-sized phantom (activity and attenuation map on the
reconstruction grid) and listmode events drawn by Monte Carlo: an emission
point sampled from the activity, an isotropic direction, the two points where
the line meets the crystal cylinder snapped to the nearest crystals, survival
of the pair against attenuation taken from the exact chord through the head
ellipsoid (water), detector-pair efficiency, plus uniformly distributed
random coincidences.  Written with torch tensor ops so that it runs on the
CPU for small test cases and on the GPU for the benchmark's full size.

Sizes follow the paper's PET example (Sec. 3.2): a 338 mm ring radius,
eight 32.25 mm ring modules (here 64 crystal rings of 4.03 mm), a
204 x 204 x 154 image of 1.25 mm voxels and a 3 mm FWHM resolution model.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

WATER_MU_MM = 0.0096   # 511 keV, 1/mm
C_MM_PER_PS = 0.299792458
FWHM_PER_SIGMA = 2.0 * math.sqrt(2.0 * math.log(2.0))
BONE_MU_MM = 0.0172


@dataclass(frozen=True)
class Scanner:
    radius_mm: float = 338.0
    crystals_per_ring: int = 448
    rings: int = 64
    ring_pitch_mm: float = 4.03125

    @property
    def n_crystals(self) -> int:
        return self.crystals_per_ring * self.rings

    @property
    def axial_half_mm(self) -> float:
        return 0.5 * self.rings * self.ring_pitch_mm

    def crystal_xyz(self, ids: torch.Tensor) -> torch.Tensor:
        ring = torch.div(ids, self.crystals_per_ring, rounding_mode="floor")
        k = ids - ring * self.crystals_per_ring
        phi = 2.0 * math.pi * k.double() / self.crystals_per_ring
        z = (ring.double() - 0.5 * (self.rings - 1)) * self.ring_pitch_mm
        return torch.stack([self.radius_mm * torch.cos(phi), self.radius_mm * torch.sin(phi), z], dim=-1)


@dataclass(frozen=True)
class PetWorkload:
    name: str
    shape: tuple
    voxel: tuple
    scanner: Scanner
    prompts: int
    randoms_frac: float
    n_subsets: int
    n_iters: int
    fwhm_mm: float
    seed: int
    tof_bins: int = 0          # time-of-flight bins (0: none)
    tof_range_mm: float = 0.0  # total extent of the bins along the line
    tof_fwhm_ps: float = 0.0   # coincidence timing resolution

    @property
    def rr_sigma_mm(self) -> float:
        return self.fwhm_mm / FWHM_PER_SIGMA

    @property
    def tof_bin_mm(self) -> float:
        return self.tof_range_mm / self.tof_bins if self.tof_bins else 0.0

    @property
    def tof_sigma_mm(self) -> float:
        # a timing difference dt moves the annihilation point by c dt / 2
        return 0.5 * C_MM_PER_PS * self.tof_fwhm_ps / FWHM_PER_SIGMA


PET_WORKLOADS = {
    # the paper's PET reconstruction grid and scanner; 3 subsets as in its
    # high-count LM OSEM; 30 M prompts
    "petlm204": PetWorkload("petlm204", (204, 204, 154), (1.25, 1.25, 1.25), Scanner(), 30_000_000, 0.1, 3, 1,
                            3.0, 11),
    # the same with the paper's time of flight: 550 ps, 21 bins over 30 cm
    "petlm204tof": PetWorkload("petlm204tof", (204, 204, 154), (1.25, 1.25, 1.25), Scanner(), 30_000_000, 0.1, 3, 1,
                               3.0, 11, 21, 300.0, 550.0),
    # a small case for parity tests
    "petlm_small": PetWorkload("petlm_small", (40, 40, 28), (3.0, 3.0, 3.5),
                               Scanner(radius_mm=110.0, crystals_per_ring=96, rings=12, ring_pitch_mm=7.5),
                               40_000, 0.1, 3, 2, 6.0, 3),
}

HEAD_SEMI_MM = (72.0, 90.0, 85.0)  # x, y, z semi-axes of the head ellipsoid
SKULL_MM = 6.0


def _grid(shape, voxel, device):
    axes = [(torch.arange(n, device=device, dtype=torch.float64) - 0.5 * (n - 1)) * v for n, v in zip(shape, voxel)]
    return torch.meshgrid(*axes, indexing="ij")


def head_phantom(shape, voxel, seed: int, device="cpu"):
    """(activity, mu) on the image grid, float32: a head ellipsoid (scaled to
    the field of view when the grid is small) with a skull shell, cortex at
    activity 4, white matter 1, ventricles 0 and five hot lesions at 8;
    mu = water inside, bone in the skull."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    x, y, z = _grid(shape, voxel, device)
    fov = [0.5 * n * v for n, v in zip(shape, voxel)]
    scale = min(1.0, min(0.9 * f / h for f, h in zip(fov, HEAD_SEMI_MM)))
    a, b, c = (h * scale for h in HEAD_SEMI_MM)
    r = torch.sqrt((x / a) ** 2 + (y / b) ** 2 + (z / c) ** 2)
    skull = SKULL_MM * scale / min(a, b, c)
    act = torch.zeros(shape, dtype=torch.float64, device=device)
    mu = torch.zeros(shape, dtype=torch.float64, device=device)
    inside = r <= 1.0
    mu[inside] = WATER_MU_MM
    mu[(r > 1.0 - skull) & inside] = BONE_MU_MM
    brain = r <= 1.0 - skull
    act[brain] = 1.0
    act[(r > 0.78 - skull) & brain] = 4.0
    vent = ((x / (0.15 * a)) ** 2 + (y / (0.35 * b)) ** 2 + ((z - 0.1 * c) / (0.25 * c)) ** 2) <= 1.0
    act[vent] = 0.0
    for _ in range(5):
        u = torch.rand(3, generator=g, dtype=torch.float64) * 2 - 1
        u = u / max(1.0, float(torch.linalg.norm(u))) * 0.55
        rad = float(torch.rand(1, generator=g, dtype=torch.float64)) * 6.0 * scale + 4.0 * scale
        d = torch.sqrt((x - u[0] * a) ** 2 + (y - u[1] * b) ** 2 + (z - u[2] * c) ** 2)
        act[d <= rad] = 8.0
    return act.float(), mu.float(), (a, b, c)


def _ellipsoid_chord(p, d, semi):
    """Length (mm) of the part of each line p + t d (t in R, |d| = 1) inside
    the ellipsoid with semi-axes `semi` centred at the origin."""
    s = torch.tensor(semi, dtype=torch.float64, device=p.device)
    ps, ds = p / s, d / s
    A = (ds * ds).sum(-1)
    B = 2.0 * (ps * ds).sum(-1)
    C = (ps * ps).sum(-1) - 1.0
    disc = torch.clamp(B * B - 4 * A * C, min=0.0)
    return torch.sqrt(disc) / A


def draw_events(wl: PetWorkload, act: torch.Tensor, semi, device="cpu", chunk: int = 20_000_000):
    """Listmode events: (lors [n][6] float32 mm, eta [n] float32, s [n]
    float32, true_count, tof_bin [n] int32 or None).  Prompts = trues +
    randoms in random order; eta is the product of the two crystals'
    efficiencies; s is the expected number of randoms on one crystal pair
    (and time-of-flight bin).  A true event's bin is its emission point's
    arc length from the line's midpoint plus Gaussian timing noise; a
    random's bin is uniform."""
    sc = wl.scanner
    gen = torch.Generator(device=device).manual_seed(wl.seed)
    cpu_gen = torch.Generator(device="cpu").manual_seed(wl.seed + 1)
    eff = (0.85 + 0.3 * torch.rand(sc.n_crystals, generator=cpu_gen, dtype=torch.float64)).to(device)
    n_rand = int(round(wl.randoms_frac * wl.prompts))
    n_true = wl.prompts - n_rand
    cdf = torch.cumsum(act.double().flatten().to(device), 0)
    cdf = cdf / cdf[-1]
    shape = torch.tensor(wl.shape, device=device)
    vox = torch.tensor(wl.voxel, dtype=torch.float64, device=device)
    half = 0.5 * (shape.double() - 1.0)
    got_a, got_b, got_l = [], [], []
    have = 0
    while have < n_true:
        m = min(chunk, max(4 * (n_true - have), 1024))
        # emission voxel by inverse transform sampling of the activity
        u = torch.rand(m, generator=gen, dtype=torch.float64, device=device)
        idx = torch.clamp(torch.searchsorted(cdf, u, right=True), max=cdf.numel() - 1)
        k = idx % wl.shape[2]
        j = torch.div(idx, wl.shape[2], rounding_mode="floor") % wl.shape[1]
        i = torch.div(idx, wl.shape[1] * wl.shape[2], rounding_mode="floor")
        ijk = torch.stack([i, j, k], dim=-1).double()
        pos = (ijk - half + torch.rand(m, 3, generator=gen, dtype=torch.float64, device=device) - 0.5) * vox
        d = torch.randn(m, 3, generator=gen, dtype=torch.float64, device=device)
        d = d / torch.linalg.norm(d, dim=-1, keepdim=True)
        # meet the crystal cylinder
        A = d[:, 0] ** 2 + d[:, 1] ** 2
        B = 2 * (pos[:, 0] * d[:, 0] + pos[:, 1] * d[:, 1])
        C = pos[:, 0] ** 2 + pos[:, 1] ** 2 - sc.radius_mm ** 2
        root = torch.sqrt(torch.clamp(B * B - 4 * A * C, min=0.0))
        A = torch.clamp(A, min=1e-300)
        t1, t2 = (-B - root) / (2 * A), (-B + root) / (2 * A)
        e1, e2 = pos + t1[:, None] * d, pos + t2[:, None] * d
        ok = (e1[:, 2].abs() < sc.axial_half_mm) & (e2[:, 2].abs() < sc.axial_half_mm)
        # survival against attenuation through the water head
        surv = torch.exp(-WATER_MU_MM * _ellipsoid_chord(pos, d, semi))
        ok &= torch.rand(m, generator=gen, dtype=torch.float64, device=device) < surv
        ca, cb = _snap(sc, e1[ok]), _snap(sc, e2[ok])
        eta = eff[ca] * eff[cb]
        keep = (torch.rand(ca.shape[0], generator=gen, dtype=torch.float64, device=device) < eta / 1.15 ** 2) & (ca != cb)
        got_a.append(ca[keep])
        got_b.append(cb[keep])
        if wl.tof_bins:
            p1, p2 = sc.crystal_xyz(ca[keep]), sc.crystal_xyz(cb[keep])
            u = (p2 - p1) / torch.linalg.norm(p2 - p1, dim=-1, keepdim=True)
            got_l.append(((pos[ok][keep] - 0.5 * (p1 + p2)) * u).sum(-1))
        have += int(keep.sum())
    ca = torch.cat(got_a)[:n_true]
    cb = torch.cat(got_b)[:n_true]
    ra = torch.randint(0, sc.n_crystals, (n_rand,), generator=gen, device=device)
    rb = (ra + torch.randint(1, sc.n_crystals, (n_rand,), generator=gen, device=device)) % sc.n_crystals
    ca, cb = torch.cat([ca, ra]), torch.cat([cb, rb])
    tof = None
    if wl.tof_bins:
        ell = torch.cat(got_l)[:n_true]
        ell = ell + wl.tof_sigma_mm * torch.randn(n_true, generator=gen, dtype=torch.float64, device=device)
        tb = torch.round(ell / wl.tof_bin_mm + 0.5 * (wl.tof_bins - 1)).long().clamp(0, wl.tof_bins - 1)
        tof = torch.cat([tb, torch.randint(0, wl.tof_bins, (n_rand,), generator=gen, device=device)])
    perm = torch.randperm(ca.shape[0], generator=gen, device=device)
    ca, cb = ca[perm], cb[perm]
    lors = torch.cat([sc.crystal_xyz(ca), sc.crystal_xyz(cb)], dim=-1).float().contiguous()
    eta = (eff[ca] * eff[cb]).float().contiguous()
    pairs = sc.n_crystals * (sc.n_crystals - 1) / 2
    s = torch.full((ca.shape[0],), n_rand / pairs / max(wl.tof_bins, 1), dtype=torch.float32, device=device)
    if tof is not None:
        tof = tof[perm].int().contiguous()
    return lors, eta, s, n_true, tof


def _snap(sc: Scanner, pts: torch.Tensor) -> torch.Tensor:
    phi = torch.atan2(pts[:, 1], pts[:, 0])
    k = torch.round(phi / (2 * math.pi) * sc.crystals_per_ring).long() % sc.crystals_per_ring
    ring = torch.round(pts[:, 2] / sc.ring_pitch_mm + 0.5 * (sc.rings - 1)).long().clamp(0, sc.rings - 1)
    return ring * sc.crystals_per_ring + k


def scanner_lors(sc: Scanner, angle_step: int = 1, ring_step: int = 1, device="cpu", eff_seed: int = None):
    """Every crystal pair (i < j) among crystals k % angle_step == 0 of rings
    r % ring_step == 0, as (lors [n][6] float32, eta [n] float32 or None,
    weight): the LOR set of the sensitivity image, each LOR standing for
    weight = (angle_step * ring_step)^2 pairs of the full scanner."""
    ks = torch.arange(0, sc.crystals_per_ring, angle_step, device=device)
    rs = torch.arange(0, sc.rings, ring_step, device=device)
    ids = (rs[:, None] * sc.crystals_per_ring + ks[None, :]).flatten()
    ia, ib = torch.triu_indices(ids.numel(), ids.numel(), offset=1, device=device)
    ca, cb = ids[ia], ids[ib]
    lors = torch.cat([sc.crystal_xyz(ca), sc.crystal_xyz(cb)], dim=-1).float().contiguous()
    eta = None
    if eff_seed is not None:
        cpu_gen = torch.Generator(device="cpu").manual_seed(eff_seed + 1)
        eff = (0.85 + 0.3 * torch.rand(sc.n_crystals, generator=cpu_gen, dtype=torch.float64)).to(device)
        eta = (eff[ca] * eff[cb]).float().contiguous()
    return lors, eta, float((angle_step * ring_step) ** 2)
