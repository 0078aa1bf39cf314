"""Geometry and material tables for the synthetic workloads (inputs only, no BEM arithmetic).

Conventions shared with the C interface (``include/bem.h``):

* Domains are numbered from 0; domain 0 is the unbounded host medium (Omega_1 of the paper, Sec. 2),
  whose flux coefficient is 1.
* A segment is a polyline ``xy`` of ``n_vert`` vertices.  A closed segment also has the element from the
  last vertex back to the first.  Element e joins vertex e to vertex e+1.
* The unit normal of an element is its tangent turned by +90 degrees (the left normal of the direction
  of travel).  It points out of domain ``P`` and into domain ``M`` (Sec. 2: on the boundary of Omega_1
  the normal is directed away from Omega_1).  So a counter-clockwise circle around a scatterer has
  ``P = 0`` (host) and ``M`` = the scatterer.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Segment:
    xy: np.ndarray          # (n_vert, 2) float64 vertices
    P: int                  # domain the normal points out of
    M: int                  # domain the normal points into
    closed: bool

    @property
    def n_elem(self) -> int:
        return len(self.xy) if self.closed else len(self.xy) - 1


@dataclass
class Problem:
    """One scattering problem: domains (wavenumber k_d, flux coefficient eps_d) and interface segments."""
    k: list
    eps: list
    segments: list = field(default_factory=list)
    name: str = ""

    @property
    def n_elem(self) -> int:
        return sum(s.n_elem for s in self.segments)

    @property
    def n_unknowns(self) -> int:
        return 2 * self.n_elem


def _closed_curve(r_of_t, n: int, phase: float = 0.0, clockwise: bool = False) -> np.ndarray:
    t = 2.0 * np.pi * np.arange(n, dtype=np.float64) / n + phase
    if clockwise:
        t = -t
    x, y = r_of_t(t)
    return np.stack([x, y], axis=1)


def circle(n: int, R: float = 1.0, center=(0.0, 0.0), clockwise: bool = False) -> np.ndarray:
    """Inscribed regular n-gon of a circle (vertices at equal angles, first vertex at angle 0)."""
    cx, cy = center
    return _closed_curve(lambda t: (cx + R * np.cos(t), cy + R * np.sin(t)), n, clockwise=clockwise)


def ellipse(n: int, aspect: float, clockwise: bool = False) -> np.ndarray:
    """Ellipse of unit area-equivalent radius: semi-axes sqrt(aspect) and 1/sqrt(aspect)."""
    a, b = math.sqrt(aspect), 1.0 / math.sqrt(aspect)
    return _closed_curve(lambda t: (a * np.cos(t), b * np.sin(t)), n, clockwise=clockwise)


def star(n: int, amp: float = 0.3, lobes: int = 5, phase: float = 0.0) -> np.ndarray:
    """Star-shaped curve r(t) = 1 + amp*cos(lobes*t + phase), vertices at equal steps of t, CCW."""
    def rt(t):
        r = 1.0 + amp * np.cos(lobes * t + phase)
        return r * np.cos(t), r * np.sin(t)
    return _closed_curve(rt, n)


def square(n_per_side: int, side: float = 1.0) -> np.ndarray:
    """Square [0,side]^2 traversed CCW with n_per_side equal elements per side."""
    s = np.linspace(0.0, side, n_per_side + 1)[:-1]
    bottom = np.stack([s, np.zeros_like(s)], 1)
    right = np.stack([np.full_like(s, side), s], 1)
    top = np.stack([side - s, np.full_like(s, side)], 1)
    left = np.stack([np.zeros_like(s), side - s], 1)
    return np.concatenate([bottom, right, top, left], 0)


def circle_problem(n: int, k_e: float, k_i: float, eps_i: float | None = None, R: float = 1.0,
                   name: str = "circle") -> Problem:
    """Single penetrable circle (Sec. 7.1).  eps_i defaults to (k_i/k_e)^2, i.e. k_i = omega*sqrt(eps_i)."""
    if eps_i is None:
        eps_i = (k_i / k_e) ** 2
    return Problem(k=[k_e, k_i], eps=[1.0, eps_i],
                   segments=[Segment(circle(n, R), P=0, M=1, closed=True)], name=name)


def concentric(n_inner: int, n_outer: int, omega: float, eps=(1.0, 2.0, 3.0),
               R_in: float = 1.0, R_out: float = 2.0) -> Problem:
    """Concentric circles of Sec. 7.2: outer ring Omega_2 (R_out), inner disk Omega_3 (R_in).

    Both normals point into Omega_2 (Sec. 6): on the outer circle from Omega_1 into Omega_2 (CCW), on the
    inner circle from Omega_3 into Omega_2 (clockwise traversal)."""
    k = [omega * math.sqrt(e) for e in eps]
    return Problem(k=k, eps=list(eps), segments=[
        Segment(circle(n_outer, R_out), P=0, M=1, closed=True),
        Segment(circle(n_inner, R_in, clockwise=True), P=2, M=1, closed=True),
    ], name="concentric")


def junction_disk(n_total: int, k=(15.0, 22.5, 30.0), eps=None) -> Problem:
    """Unit disk split by the diameter x_1 = 0 into two materials; two triple junctions at (0, +-1).

    Domain 1 is the left half, domain 2 the right half.  Each arc carries 3/8 of the elements and the
    diameter 1/4 (the arc/chord split of Sec. 7.2).  Arc normals point into the disk; the diameter normal
    points from the right half (domain 2) into the left half (domain 1)."""
    if eps is None:
        eps = [1.0] + [(kk / k[0]) ** 2 for kk in k[1:]]
    n_dia = n_total // 4
    n_arc = (n_total - n_dia) // 2
    n_dia = n_total - 2 * n_arc
    ta = np.pi / 2 + np.pi * np.arange(n_arc + 1) / n_arc            # left arc, CCW from (0,1) to (0,-1)
    left = np.stack([np.cos(ta), np.sin(ta)], 1)
    tb = -np.pi / 2 + np.pi * np.arange(n_arc + 1) / n_arc           # right arc, CCW from (0,-1) to (0,1)
    right = np.stack([np.cos(tb), np.sin(tb)], 1)
    ys = -1.0 + 2.0 * np.arange(n_dia + 1) / n_dia                   # diameter, upward: left normal = -x
    dia = np.stack([np.zeros_like(ys), ys], 1)
    left[0] = (0.0, 1.0); left[-1] = (0.0, -1.0)
    right[0] = (0.0, -1.0); right[-1] = (0.0, 1.0)
    return Problem(k=list(k), eps=list(eps), segments=[
        Segment(left, P=0, M=1, closed=False),
        Segment(right, P=0, M=2, closed=False),
        Segment(dia, P=2, M=1, closed=False),
    ], name="junction_disk")


def plane_wave_angles(n: int) -> np.ndarray:
    """n incident directions uniform on [0, 2*pi)."""
    return 2.0 * np.pi * np.arange(n, dtype=np.float64) / n


# ---------------------------------------------------------------------------------------------
# The five benchmark workloads.
# ---------------------------------------------------------------------------------------------

def cfg_circle_c1(n: int = 256) -> Problem:
    """Penetrable unit circle, k_e = 5, k_i = 7.5 (refractive index 1.5), 256 elements."""
    return circle_problem(n, 5.0, 7.5, name="circle_k5_n256")


def cfg_star_c2(n: int = 4096) -> Problem:
    """Star r(t) = 1 + 0.3 cos(5t), k_e = 20, k_i = 30, 4096 elements."""
    return Problem(k=[20.0, 30.0], eps=[1.0, 2.25],
                   segments=[Segment(star(n, 0.3, 5), P=0, M=1, closed=True)], name=f"star5_k20_n{n}")


def cfg_junction_c3(n: int = 8192) -> Problem:
    """Junction disk: host k = 15, halves k = 22.5 and k = 30, 8192 elements."""
    return junction_disk(n, k=(15.0, 22.5, 30.0))


def cfg_random_stars_c4(count: int = 256, seed: int = 2312, n_min: int = 128, n_max: int = 2048):
    """Independent random stars: 3..7 lobes, amplitude U[0.1,0.4], N_e ~ U[n_min,n_max], k_e ~ U[1,40],
    contrast n ~ U[1.2,2.0] (k_i = n*k_e, eps = n^2)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(rng.integers(3, 8))
        amp = float(rng.uniform(0.1, 0.4))
        ph = float(rng.uniform(0.0, 2 * np.pi))
        ne = int(rng.integers(n_min, n_max + 1))
        ke = float(rng.uniform(1.0, 40.0))
        nc = float(rng.uniform(1.2, 2.0))
        out.append(Problem(k=[ke, nc * ke], eps=[1.0, nc * nc],
                           segments=[Segment(star(ne, amp, m, ph), P=0, M=1, closed=True)],
                           name=f"star{m}_{i}"))
    return out


def cfg_omega_eps_sweep(n: int = 600, count: int = 64):
    """The single-material iteration study of Sec. 7.1 as one workload: the unit circle of n elements,
    (a) `count` angular frequencies omega in [0.5, 20] with eps_2 = 2, and (b) `count` contrasts eps_2 in
    [1.1, 10] with omega = 5.  The paper plots both (ranges read off its setting; the text gives none), for the
    proposed and the conventional arrangement.  Returns [(label, value, Problem)]."""
    out = []
    for w in np.linspace(0.5, 20.0, count):
        out.append(("omega", float(w), circle_problem(n, w, w * math.sqrt(2.0), eps_i=2.0, name=f"circle_w{w:.3f}")))
    for e in np.linspace(1.1, 10.0, count):
        out.append(("eps", float(e), circle_problem(n, 5.0, 5.0 * math.sqrt(e), eps_i=float(e), name=f"circle_e{e:.3f}")))
    return out


def cfg_concentric_sweep(n_inner: int = 600, n_outer: int = 1200, count: int = 32):
    """The concentric iteration study of Sec. 7.2: (a) `count` angular frequencies omega in [0.5, 10] with
    eps_i = i, and (b) `count` contrasts eps_2 = 1/eps_3 for eps_3 in [0.1, 10] with omega = 5, on the inner
    and outer circles of n_inner and n_outer elements (ranges read off the setting; the text gives none).
    Returns [(label, value, Problem)]."""
    out = []
    for w in np.linspace(0.5, 10.0, count):
        out.append(("omega", float(w), concentric(n_inner, n_outer, float(w), eps=(1.0, 2.0, 3.0))))
    for e3 in np.linspace(0.1, 10.0, count):
        out.append(("eps", float(e3), concentric(n_inner, n_outer, 5.0, eps=(1.0, 1.0 / float(e3), float(e3)))))
    return out


def cfg_serving_c5(count: int = 2000, seed: int = 2313, rate: float = 200.0,
                   n_min: int = 256, n_max: int = 16384):
    """Poisson request stream mixing circles, ellipses (aspect U[1,4]) and two-material junction disks.

    Returns a list of (arrival_time_s, Problem).  N_e is log-uniform on [n_min, n_max], k_e ~ U[1,50],
    contrast ~ U[1.2,2.0]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        kind = int(rng.integers(0, 3))
        ne = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        ke = float(rng.uniform(1.0, 50.0))
        nc = float(rng.uniform(1.2, 2.0))
        if kind == 0:
            p = Problem(k=[ke, nc * ke], eps=[1.0, nc * nc],
                        segments=[Segment(circle(ne), P=0, M=1, closed=True)], name=f"circle_{i}")
        elif kind == 1:
            asp = float(rng.uniform(1.0, 4.0))
            p = Problem(k=[ke, nc * ke], eps=[1.0, nc * nc],
                        segments=[Segment(ellipse(ne, asp), P=0, M=1, closed=True)], name=f"ellipse_{i}")
        else:
            nc2 = float(rng.uniform(1.2, 2.0))
            p = junction_disk(max(ne, 16), k=(ke, nc * ke, nc2 * ke))
            p.name = f"junction_{i}"
        out.append((t, p))
    return out


def junction_material(n_total: int, omega: float, eps2: float, eps3: float) -> Problem:
    """The junction disk of Sec. 7.2 with k_d = omega sqrt(eps_d): host eps_1 = 1, left half eps_2, right half
    eps_3 (domains 1 and 2 here), 3/4 of the elements on the circle and 1/4 on the diameter."""
    return junction_disk(n_total, k=(omega, omega * math.sqrt(eps2), omega * math.sqrt(eps3)),
                         eps=(1.0, eps2, eps3))


def cfg_junction_sweep(n_fixed: int = 1066, n_values=(266, 400, 533, 800, 1066, 1600, 2132, 3198),
                       count: int = 32):
    """The junction-scatterer iteration study of Sec. 7.2 (three materials meeting at two points): the same
    sweeps as the concentric study on the junction disk, (a) over the number of elements N with eps_i = i and
    omega = 5 (the N values are a choice), (b) `count` angular frequencies omega in [0.5, 10] with eps_i = i at
    N = n_fixed, and (c) `count` contrasts eps_2 = 1/eps_3 for eps_3 in [0.1, 10] with omega = 5 at N = n_fixed
    (the paper fixes N = 1066 for (b) and (c); the omega and eps ranges are read off its setting).
    Returns [(label, value, Problem)]."""
    out = []
    for n in n_values:
        out.append(("n", float(n), junction_material(int(n), 5.0, 2.0, 3.0)))
    for w in np.linspace(0.5, 10.0, count):
        out.append(("omega", float(w), junction_material(n_fixed, float(w), 2.0, 3.0)))
    for e3 in np.linspace(0.1, 10.0, count):
        out.append(("eps", float(e3), junction_material(n_fixed, 5.0, 1.0 / float(e3), float(e3))))
    return out

