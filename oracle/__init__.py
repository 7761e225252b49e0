"""FP64 CPU oracle for the color-gradient LBM step (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use this package. It never imports the CUDA library or its binding, and
the CUDA path never imports it.

Parity status of each oracle function (what pins it, see ``tests/test_oracle_*``):
  * lattice tables, M and M^-1      closed forms (isotropy sums, orthogonality)
  * indexer                         brute force (set-based re-derivation) and
                                    neighbour symmetry
  * collision                       fixed point, BGK special case, conservation
  * recoloring                      conservation, beta cancellation, A/B symmetry
  * gradient                        exact on linear and quadratic fields, phi_s
  * streaming + bounce-back         unit pulse, mass conservation, dense np.roll
                                    brute force on 8^3
  * full model                      duct Poiseuille series, flat-interface tanh
                                    profile, Laplace law (sigma = 6 alpha),
                                    contact angle cos(theta) = phi_s
  * reservoir slabs                 exact reset state after every step; with
                                    equal reservoir densities the closed-form
                                    steady state (rest, linear component
                                    densities); saturation rising monotonically
                                    and the front advancing under injection
  * pressure faces, flux inlet      exact face density and zero tangential
                                    momentum, pressure-driven and flux-driven
                                    duct series, uniform component density
                                    between two faces at equal density
  * the pins themselves             planted mistakes in copies of this oracle
                                    each fail a named pin
"""
from .core import (  # noqa: F401
    Oracle,
    lattice_check,
    lattice_tables,
    collide_site,
    recolor_site,
    load_library,
    MEASURE_FIELDS,
    set_threads,
    get_threads,
    have_openmp,
)
