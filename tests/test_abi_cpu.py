"""CPU checks of the C ABI: the library builds, loads and exports every
function include/spect.h and include/pet.h declare; host-side validation
rejects bad geometry before touching the GPU.  No kernel runs here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fname in os.listdir(os.path.join(ROOT, "include")):
        if not fname.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fname)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][A-Za-z0-9_ ]*[\s*]+((?:spect|pet)_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("spect_plan_create", "spect_forward", "spect_back", "spect_osem_run", "spect_sensitivity"):
        assert required in names


def test_library_exports_every_declared_symbol(spect_lib):
    lib = ctypes.CDLL(spect_lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(spect_lib.EXPORTED) <= set(declared_functions())
    from paper_2309_01977_gb300 import pet
    assert set(pet.PET_EXPORTED) == {n for n in declared_functions() if n.startswith("pet_")}


def test_status_strings(spect_lib):
    lib = spect_lib.load()
    assert lib.spect_status_str(0) == b"SPECT_OK"
    assert lib.spect_status_str(-1) == b"SPECT_EINVAL"
    assert lib.spect_status_str(-5) == b"SPECT_ETIMEDOUT"
    assert lib.spect_status_str(-99) == b"SPECT_UNKNOWN"
    assert b"sm_103a" in lib.spect_version()


@pytest.mark.parametrize("bad, msg", [
    (dict(n=16, nz=18), "nz"),
    (dict(n=1, nz=16), "nx"),
    (dict(n=16, nz=16, n_angles=0), "n_angles"),
    (dict(n=16, nz=16, n_subsets=0), "n_subsets"),
    (dict(n=16, nz=16, n_subsets=40), "n_subsets"),
    (dict(n=16, nz=16, psf_sigma0=-1.0), "PSF"),
    (dict(n=16, nz=16, psf_nsigma=0.0), "PSF"),
])
def test_geometry_validation(spect_lib, bad, msg):
    kw = dict(n=16, nz=16, n_angles=12, n_subsets=3, attenuation=False)
    kw.update(bad)
    g = spect_lib.Geometry(**kw)
    with pytest.raises(spect_lib.SpectError) as e:
        spect_lib.spect_plan_create(g, None, stream=0)
    assert e.value.status == spect_lib.SPECT_EINVAL
    assert msg in str(e.value)


def test_nonsquare_and_missing_mu_rejected(spect_lib):
    lib = spect_lib.load()
    g, _ = spect_lib.Geometry(n=16, nz=16, n_angles=4, attenuation=True).to_c()
    out = ctypes.c_void_p()
    assert lib.spect_plan_create(ctypes.byref(g), None, None, ctypes.byref(out)) == spect_lib.SPECT_EINVAL
    assert b"mu" in lib.spect_last_error()
    g.ny = 17
    assert lib.spect_plan_create(ctypes.byref(g), None, None, ctypes.byref(out)) == spect_lib.SPECT_EINVAL
    assert out.value is None


def test_null_plan_rejected(spect_lib):
    lib = spect_lib.load()
    assert lib.spect_forward(None, None, None, 0, 1, None) == spect_lib.SPECT_EINVAL
    assert lib.spect_osem_run(None, None, ctypes.c_float(0.0), None, 0, 1, None, None) == spect_lib.SPECT_EINVAL
    assert lib.spect_plan_destroy(None) == 0


def test_serve_config_validation(spect_lib):
    lib = spect_lib._serve_lib()
    out = ctypes.c_void_p()
    for cfg in [(0, 4, 4, 1000), (1 << 30, 0, 4, 1000), (1 << 30, 4, 0, 1000), (1 << 30, 4, 4, 0)]:
        c = spect_lib._ServeCfg(*cfg)
        assert lib.spect_serve_create(ctypes.byref(c), ctypes.byref(out)) == spect_lib.SPECT_EINVAL
        assert out.value is None
    rid = ctypes.c_uint64()
    assert lib.spect_serve_submit(None, None, ctypes.byref(rid)) == spect_lib.SPECT_EINVAL
    st = ctypes.c_int()
    assert lib.spect_serve_poll(None, 1, ctypes.byref(st)) == spect_lib.SPECT_EINVAL
    assert lib.spect_serve_destroy(None) == 0


@pytest.mark.parametrize("bad, msg", [
    (dict(shape=(0, 4, 4)), "image size"),
    (dict(voxel=(1.0, 0.0, 1.0)), "voxel"),
    (dict(n_subsets=0), "n_subsets"),
    (dict(rr_sigma_mm=2.0, rr_nsigma=0.0), "rr_nsigma"),
    (dict(rr_sigma_mm=40.0), "radius"),
    (dict(n_tof_bins=-1), "n_tof_bins"),
    (dict(n_tof_bins=5, tof_bin_mm=10.0), "time of flight"),
])
def test_pet_geometry_validation(spect_lib, bad, msg):
    from paper_2309_01977_gb300 import pet
    kw = dict(shape=(8, 8, 8), voxel=(2.0, 2.0, 2.0))
    kw.update(bad)
    g = pet.PetGeometry(**kw).to_c()
    out = ctypes.c_void_p()
    lib = pet.load()
    assert lib.pet_plan_create(ctypes.byref(g), None, None, ctypes.byref(out)) == spect_lib.SPECT_EINVAL
    assert msg.encode() in lib.spect_last_error()
    assert out.value is None


def test_pet_null_plan_rejected(spect_lib):
    from paper_2309_01977_gb300 import pet
    lib = pet.load()
    assert lib.pet_forward(None, None, None, None, None, 0, None, None) == spect_lib.SPECT_EINVAL
    assert lib.pet_lm_osem_run(None, None, None, None, None, 0, None, None, 0, 1, None, None) == spect_lib.SPECT_EINVAL
