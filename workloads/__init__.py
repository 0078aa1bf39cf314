"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This package only generates input data: polygon vertices, the domain table (wavenumbers and flux
coefficients) and incident angles.  It holds none of the boundary-element arithmetic; both the
CUDA library and the CPU oracle derive elements, normals, quadrature and matrices on their own.
"""
from .geometry import (  # noqa: F401
    Problem, Segment, circle, ellipse, star, square, concentric, junction_disk,
    cfg_circle_c1, cfg_star_c2, cfg_junction_c3, cfg_random_stars_c4, cfg_serving_c5, cfg_omega_eps_sweep,
    cfg_concentric_sweep, cfg_junction_sweep, junction_material,
    circle_problem, plane_wave_angles,
)
