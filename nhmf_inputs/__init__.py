"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the finite-element method: it only draws random
numbers and describes workloads (mesh size, degree, material constants, boundary
preset, seeds).  Both the CUDA path and the CPU oracle receive the arrays it makes.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written here from its published
definition as a counter-based stream: output k (k = 0, 1, ...) of seed s is
mix(s + (k + 1) * 0x9E3779B97F4A7C15).  Uniforms are (x >> 11) * 2^-53; normals use
the Box-Muller transform on consecutive pairs of uniforms.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+count-1 of the splitmix64 stream started at `seed`."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, count: int) -> np.ndarray:
    """count doubles in [0, 1) with 53 random bits each."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm(seed: int, count: int, a: float) -> np.ndarray:
    """count doubles uniform on [-a, a)."""
    return a * (2.0 * uniform01(seed, count) - 1.0)


def normal(seed: int, count: int) -> np.ndarray:
    """count standard normal doubles (Box-Muller on consecutive uniform pairs)."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1, u2 = 1.0 - u[0::2], u[1::2]          # 1 - u1 lies in (0, 1]: log is finite
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


# Boundary presets: 0 none, 1 clamp the face x = 0, 2 compression (clamp z = 0, prescribe
# u_z on z = 1, u_x and u_y free there).
BC_NONE, BC_CLAMP_X0, BC_COMPRESSION = 0, 1, 2


@dataclass(frozen=True)
class Workload:
    name: str
    n_el: int                 # elements per direction of the unit cube
    degree: int               # polynomial degree p of Q_p
    mu: float
    lam: float
    bc: int
    u_rule: str               # "literal": u ~ U(-a, a); "scaled": u = (h/p) U(-a, a)
    u_amp: float
    du_rule: str              # "uniform": U(-du_amp, du_amp); "normal": N(0, 1)
    du_amp: float
    seed_u: int
    seed_du: int
    load_steps: int = 0       # compression presets: number of load steps
    compression: float = 0.0  # total top-face z displacement magnitude

    @property
    def n_nodes_1d(self) -> int:
        return self.degree * self.n_el + 1

    @property
    def n_dofs(self) -> int:
        return 3 * self.n_nodes_1d ** 3

    @property
    def n_elements(self) -> int:
        return self.n_el ** 3

    @property
    def n_qp(self) -> int:
        return self.n_elements * (self.degree + 1) ** 3


WORKLOADS = {
    # Q1 8^3, clamp x = 0, literal U(+-0.01) draws for u and du.
    "q1_8_clamp": Workload("q1_8_clamp", 8, 1, 1.0, 1.5, BC_CLAMP_X0, "literal", 0.01,
                           "uniform", 0.01, 1001, 2001),
    # Q2 64^3 and Q4 32^3: u = (h/p) U(+-0.05), du ~ N(0, 1), clamp x = 0.
    "q2_64_clamp": Workload("q2_64_clamp", 64, 2, 1.0, 1.5, BC_CLAMP_X0, "scaled", 0.05,
                            "normal", 1.0, 1002, 2002),
    "q4_32_clamp": Workload("q4_32_clamp", 32, 4, 1.0, 1.5, BC_CLAMP_X0, "scaled", 0.05,
                            "normal", 1.0, 1002, 2002),
    # Q3 48^3 near-incompressible compression, 10 load steps of 1 %.
    "q3_48_compress": Workload("q3_48_compress", 48, 3, 1.0, 49.0, BC_COMPRESSION, "scaled", 0.05,
                               "normal", 1.0, 1003, 2003, load_steps=10, compression=0.1),
    # Q2 64^3 compression, 20 load steps, nu = 0.3 labelling.
    "q2_64_compress": Workload("q2_64_compress", 64, 2, 1.0, 1.5, BC_COMPRESSION, "scaled", 0.05,
                               "normal", 1.0, 1004, 2004, load_steps=20, compression=0.1),
    # Q4 64^3 near-incompressible, 51 M DoFs.
    "q4_64_compress": Workload("q4_64_compress", 64, 4, 1.0, 49.0, BC_COMPRESSION, "scaled", 0.05,
                               "normal", 1.0, 1005, 2005, load_steps=10, compression=0.1),
}


def small(w: Workload, n_el: int, degree: int | None = None) -> Workload:
    """The same recipe on a smaller mesh (and optionally another degree)."""
    return replace(w, name=f"{w.name}@{n_el}", n_el=n_el,
                   degree=w.degree if degree is None else degree)


def dirichlet_mask(n_el: int, degree: int, bc: int) -> np.ndarray:
    """Boolean [3, M^3] mask of constrained DoFs, DoF layout c*M^3 + i + M*(j + M*k)."""
    m = degree * n_el + 1
    mask = np.zeros((3, m, m, m), dtype=bool)          # indexed [c, k, j, i]
    if bc == BC_CLAMP_X0:
        mask[:, :, :, 0] = True
    elif bc == BC_COMPRESSION:
        mask[:, 0, :, :] = True
        mask[2, m - 1, :, :] = True
    return mask.reshape(3, m ** 3)


def draw_u(w: Workload) -> np.ndarray:
    """Linearisation point u as a flat [3*M^3] float64 array, zero on constrained DoFs."""
    n = w.n_dofs
    xi = uniform_pm(w.seed_u, n, w.u_amp)
    if w.u_rule == "scaled":
        xi *= (1.0 / w.n_el) / w.degree
    xi[dirichlet_mask(w.n_el, w.degree, w.bc).reshape(-1)] = 0.0
    return xi


def draw_du(w: Workload) -> np.ndarray:
    """Direction du as a flat [3*M^3] float64 array, zero on constrained DoFs."""
    n = w.n_dofs
    d = uniform_pm(w.seed_du, n, w.du_amp) if w.du_rule == "uniform" else normal(w.seed_du, n)
    d[dirichlet_mask(w.n_el, w.degree, w.bc).reshape(-1)] = 0.0
    return d


def draw_vector(seed: int, n: int) -> np.ndarray:
    """A plain N(0, 1) vector (test directions, right-hand sides)."""
    return normal(seed, n)


def inclusion_factors(n_el: int, stiffness: float = 100.0) -> np.ndarray:
    """Per-element material factors [N^3] (element ex + N (ey + N ez)) of a unit cube with two
    spherical inclusions `stiffness` times stiffer than the matrix (centres (0.3, 0.5, 0.5) and
    (0.7, 0.5, 0.5), radius 0.15, decided at element centres): a structured stand-in for the
    heterogeneous plate with two stiff inclusions of the paper's test case."""
    h = 1.0 / n_el
    c = (np.arange(n_el) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    f = np.ones((n_el, n_el, n_el))
    for cx in (0.3, 0.7):
        f[(x - cx) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2 <= 0.15 ** 2] = stiffness
    return f.reshape(-1)
