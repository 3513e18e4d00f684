"""FP64 CPU oracle for the SPECT and listmode PET system matrices and OSEM
(test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never imports it and
shares no code with it.  See ``spect_oracle.c`` and ``pet_oracle.c`` (front
end ``oracle.pet``) for the definitions and the readings taken where the
paper is silent.
"""
from .oracle import (  # noqa: F401
    ALGORITHMS,
    PRIORS,
    Geom,
    attenuation,
    back,
    build,
    forward,
    map_recon,
    n_threads,
    osem,
    osem_multi,
    poisson_ll,
    prior_grad,
    prior_value,
    psf_rmax,
    psf_taps,
    rotate,
    rotate_adjoint,
    set_threads,
    subset_angles,
)
