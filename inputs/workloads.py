"""Seeded synthetic inputs shared by the oracle, the CUDA path, the tests and the bench.

This module holds *inputs only*: material data in the paper's "format 1"
layout (omega, DOS, V_g, delta-omega, tau; Sec. 4.1 "Material data") built
from an isotropic Born-von Karman dispersion with a Holland-type relaxation
time, plus geometry / run descriptors for the five workloads.  None of the
Monte Carlo method's arithmetic (heat capacity from dE/dT, source energies,
alias tables, tracing, tallies) lives here; the oracle and the CUDA library
each compute those from these inputs on their own.

Units are SI at this boundary (m, s, m/s, K).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence

import numpy as np

# Face order of the paper's Boundary_prop.txt (Sec. 4.3): IDs 1..6 are
# y=0, x=Lx, y=Ly, x=0, z=0, z=Lz.  Index 0..5 below follows that order.
FACE_Y0, FACE_XL, FACE_YL, FACE_X0, FACE_Z0, FACE_ZL = range(6)
ISOTHERMAL, ADIABATIC, PERIODIC = 0, 1, 2

SI_LATTICE_A = 5.43e-10          # m, silicon lattice constant
LA_OMEGA_MAX = 7.7e13            # rad/s
TA_OMEGA_MAX = 2.8e13            # rad/s
HOLLAND_A = 1.32e-45             # s^3
HOLLAND_B = 1.73e-19             # s/K
HOLLAND_C = 137.0                # K


@dataclass
class Material:
    """Per-bin material table (paper's mat_data.txt, format 1 or 2)."""
    omega: np.ndarray            # rad/s
    v: np.ndarray                # m/s, group velocity magnitude
    tau: np.ndarray              # s, relaxation time
    D: Optional[np.ndarray] = None       # s/(rad m^3), density of states (format 1)
    domega: Optional[np.ndarray] = None  # rad/s, bin width (format 1)
    C: Optional[np.ndarray] = None       # J/(m^3 K), per-bin heat capacity (format 2)
    T_lin: float = 300.0
    name: str = ""
    tau_imp: Optional[np.ndarray] = None  # s, optional two-phonon (impurity) relaxation times
    spec_bin: Optional[np.ndarray] = None  # optional per-bin specularity d(omega) in [0, 1]

    @property
    def n_bins(self) -> int:
        return int(self.omega.shape[0])

    def scaled_tau(self, log_scale: np.ndarray) -> "Material":
        """Same material with tau_i multiplied by exp(log_scale_i)."""
        return replace(self, tau=self.tau * np.exp(np.asarray(log_scale, dtype=np.float64)))


def bvk_holland(T: float = 300.0, n_per_branch: int = 1000,
                a: float = SI_LATTICE_A) -> Material:
    """Silicon-like isotropic BvK dispersion omega = omega_max sin(pi k / 2 k_max),
    one LA and two TA branches (listed separately), uniform frequency bins with
    midpoint centres, Holland-type 1/tau = A w^4 + B w^2 T exp(-C/T).

    k_max = 2 pi / a.  The density of states per branch is the isotropic
    k^2 / (2 pi^2 v) (Eq. DOS, read with the 3-D 2 pi^2 normalisation)."""
    kmax = 2.0 * math.pi / a
    omegas, vs, Ds, dws, taus = [], [], [], [], []
    for wmax in (LA_OMEGA_MAX, TA_OMEGA_MAX, TA_OMEGA_MAX):
        dw = wmax / n_per_branch
        w = (np.arange(n_per_branch, dtype=np.float64) + 0.5) * dw
        k = (2.0 * kmax / math.pi) * np.arcsin(w / wmax)
        v = wmax * (math.pi / (2.0 * kmax)) * np.cos(math.pi * k / (2.0 * kmax))
        D = k * k / (2.0 * math.pi ** 2 * v)
        inv_tau = HOLLAND_A * w ** 4 + HOLLAND_B * w ** 2 * T * math.exp(-HOLLAND_C / T)
        omegas.append(w); vs.append(v); Ds.append(D); dws.append(np.full_like(w, dw))
        taus.append(1.0 / inv_tau)
    return Material(omega=np.concatenate(omegas), v=np.concatenate(vs),
                    tau=np.concatenate(taus), D=np.concatenate(Ds),
                    domega=np.concatenate(dws), T_lin=T, name=f"bvk_holland_{T:g}K")


def gray(v: float, mfp: float, C: float = 1.0e6, omega: float = 1.0e13,
         T: float = 300.0) -> Material:
    """Single-mode (gray) material in format 2: v, tau = mfp / v, nominal C."""
    return Material(omega=np.array([omega]), v=np.array([float(v)]),
                    tau=np.array([mfp / v]), C=np.array([float(C)]), T_lin=T,
                    name=f"gray_v{v:g}_mfp{mfp:g}")


@dataclass
class Geometry:
    """Axis-aligned box [0,Lx]x[0,Ly]x[0,Lz] (corner at origin, Sec. 4.2) with
    six faces in the paper's ID order, an optional cylindrical pore along z at
    (cx, cy), a uniform control gradient grad_T and an optional initial
    Gaussian hot spot."""
    L: Sequence[float]
    face_type: Sequence[int]
    face_T: Sequence[float] = (0.0,) * 6        # isothermal wall temperature (K)
    face_p: Sequence[float] = (0.0,) * 6        # adiabatic specularity
    T_eq: float = 300.0
    grad_T: Sequence[float] = (0.0, 0.0, 0.0)   # K/m
    pore: bool = False
    pore_c: Sequence[float] = (0.0, 0.0)
    pore_r: float = 0.0
    pore_p: float = 0.0
    gauss: bool = False
    gauss_c: Sequence[float] = (0.0, 0.0, 0.0)
    gauss_sigma: float = 0.0
    gauss_dT: float = 0.0
    # internal boundaries (Sec. 4.2): segments (x1, y1, x2, y2) in m in the x-y
    # plane through the thickness, unit normals (nx, ny) into the solid, and
    # specularities (< 0: the material's per-bin specularity)
    inner: Sequence[Sequence[float]] = ()
    inner_n: Sequence[Sequence[float]] = ()
    inner_p: Sequence[float] = ()


def slab_z(L: float, T_hot: float, T_cold: float, T_eq: float = 300.0,
           lateral: float = 100e-9) -> Geometry:
    """Cross-plane slab: isothermal z=0 (T_hot) and z=L (T_cold), periodic x, y."""
    ft = [PERIODIC] * 6
    ft[FACE_Z0] = ISOTHERMAL
    ft[FACE_ZL] = ISOTHERMAL
    fT = [0.0] * 6
    fT[FACE_Z0] = T_hot
    fT[FACE_ZL] = T_cold
    return Geometry(L=(lateral, lateral, L), face_type=ft, face_T=fT, T_eq=T_eq)


def film(d: float, W: float = 100e-9, p: float = 0.0, grad_y: float = -1.0e6,
         T_eq: float = 300.0) -> Geometry:
    """In-plane film: periodic x, y; adiabatic z faces with specularity p;
    control gradient along y."""
    ft = [PERIODIC] * 6
    ft[FACE_Z0] = ADIABATIC
    ft[FACE_ZL] = ADIABATIC
    fp = [0.0] * 6
    fp[FACE_Z0] = p
    fp[FACE_ZL] = p
    return Geometry(L=(W, W, d), face_type=ft, face_p=fp, T_eq=T_eq,
                    grad_T=(0.0, grad_y, 0.0))


def pore_lattice(W: float, porosity: float, thickness: float, p_pore: float = 0.0,
                 p_faces: float = 0.0, grad_y: float = -1.0e6,
                 T_eq: float = 300.0) -> Geometry:
    """Square lattice unit cell W x W with a cylindrical pore at the centre."""
    g = film(thickness, W=W, p=p_faces, grad_y=grad_y, T_eq=T_eq)
    g.pore = True
    g.pore_c = (0.5 * W, 0.5 * W)
    g.pore_r = W * math.sqrt(porosity / math.pi)
    g.pore_p = p_pore
    return g


def pore_skew(W: float = 100e-9, porosity: float = 0.25, thickness: float = 200e-9) -> Geometry:
    """Nanoporous cell without symmetry: the pore off centre at (0.3 W, 0.62 W)
    and the control gradient along (-0.5, -1, 0) x 1e6 K/m, diagonal in the
    film plane."""
    g = pore_lattice(W, porosity, thickness)
    g.pore_c = (0.3 * W, 0.62 * W)
    g.grad_T = (-0.5e6, -1.0e6, 0.0)
    return g


def nanomesh(W: float = 34e-9, pore: float = 11e-9, thickness: float = 22e-9, p_pore: float = 0.0,
             p_faces: float = 0.0, grad_y: float = -1.0e6, T_eq: float = 300.0) -> Geometry:
    """Square-pore nanomesh unit cell of Sec. 5.5: W x W, periodic in x and y,
    a square pore of side `pore` at the centre through the thickness, given as
    four internal walls with normals pointing away from the pore."""
    g = film(thickness, W=W, p=p_faces, grad_y=grad_y, T_eq=T_eq)
    a, b = 0.5 * (W - pore), 0.5 * (W + pore)
    g.inner = [(a, a, b, a), (b, a, b, b), (b, b, a, b), (a, b, a, a)]
    g.inner_n = [(0.0, -1.0), (1.0, 0.0), (0.0, 1.0), (-1.0, 0.0)]
    g.inner_p = [p_pore] * 4
    return g


def adiabatic_box(L: Sequence[float], p: float = 0.0, T_eq: float = 300.0) -> Geometry:
    return Geometry(L=tuple(L), face_type=[ADIABATIC] * 6, face_p=[p] * 6, T_eq=T_eq)


@dataclass
class SteadyRun:
    n: int
    seed: int
    n_cells: int = 0
    cell_axis: int = 2
    tally_axis: int = 2
    per_bin: bool = False
    n_scat_max: int = 0
    max_events: int = 10 ** 9
    # steady detector regions (Sec. 4.5): ((xmin, xmax, ymin, ymax, zmin, zmax) m, (nx, ny, nz))
    regions: Sequence = ()


@dataclass
class TransientRun:
    n: int
    seed: int
    t_max: float
    t_meas: np.ndarray
    grid: Sequence[int]
    max_events: int = 10 ** 9
    # detector regions (Sec. 4.5): ((xmin, xmax, ymin, ymax, zmin, zmax) m, (nx, ny, nz));
    # empty: the whole box split by `grid`
    regions: Sequence = ()
    # False: snapshots at each t_m (Eq. sampling); True: averages over [t_{m-1}, t_m)
    time_average: bool = False


@dataclass
class Workload:
    name: str
    material: Material
    geometries: List[Geometry]
    run: object
    n_per_geom: Optional[List[int]] = None
    notes: str = ""


def gray_slab_c1(n: int = 100_000) -> Workload:
    """Gray cross-plane slab, Kn = 1: v=6000 m/s, mfp=100 nm, L=100 nm,
    walls at T0 +/- 0.5 K, 50 cells."""
    return Workload("gray_slab_L100nm_mfp100nm", gray(6000.0, 100e-9),
                    [slab_z(100e-9, 300.5, 299.5)],
                    SteadyRun(n=n, seed=1001, n_cells=50, cell_axis=2, tally_axis=2))


def si_slab_c2(n: int = 10_000_000, material: Optional[Material] = None) -> Workload:
    """Silicon-like cross-plane film L=1 um (a 1 um cube, periodic x, y),
    3000 bins, per-bin flux tallies."""
    return Workload("si_slab_L1um_3000bins", material or bvk_holland(),
                    [slab_z(1e-6, 300.5, 299.5, lateral=1e-6)],
                    SteadyRun(n=n, seed=1002, n_cells=50, cell_axis=2, tally_axis=2,
                              per_bin=True))


def transient_box_c3(n: int = 100_000_000, grid=(64, 64, 32), n_times: int = 200,
                     material: Optional[Material] = None) -> Workload:
    """2x2x1 um adiabatic diffuse box, Gaussian +1 K (sigma 100 nm) centred on
    the top face centre, snapshots t_m = m * 10 ps, m = 1..200."""
    g = adiabatic_box((2e-6, 2e-6, 1e-6))
    g.gauss = True
    g.gauss_c = (1e-6, 1e-6, 1e-6)
    g.gauss_sigma = 100e-9
    g.gauss_dT = 1.0
    dt = 2e-9 / n_times
    t = dt * np.arange(1, n_times + 1, dtype=np.float64)
    return Workload("transient_box_2x2x1um_gauss", material or bvk_holland(), [g],
                    TransientRun(n=n, seed=1003, t_max=float(t[-1]), t_meas=t,
                                 grid=tuple(grid)))


def film_batch_c4(scale: float = 1.0, n_films: int = 64,
                  material: Optional[Material] = None) -> Workload:
    """64 in-plane films, d_f = 10 nm * 1000^(f/63), periodic x, y, diffuse z,
    grad_T = -1e6 K/m along y, N_f = round(1e5 * 100^u_f) with u_f uniform
    (numpy PCG64 seeded 1004), N_scat_max = 10.  `scale` multiplies every N_f."""
    rng = np.random.default_rng(1004)
    u = rng.uniform(0.0, 1.0, size=n_films)
    n_f = [max(1, int(round(scale * 1e5 * 100.0 ** x))) for x in u]
    ds = [10e-9 * 1000.0 ** (f / max(1, n_films - 1)) for f in range(n_films)]
    return Workload("film_batch_64_10nm_10um", material or bvk_holland(),
                    [film(d) for d in ds],
                    SteadyRun(n=0, seed=1004, tally_axis=1, per_bin=True, n_scat_max=10),
                    n_per_geom=n_f)


def pore_film_c5(n: int = 50_000_000, p_pore: float = 0.0,
                 material: Optional[Material] = None) -> Workload:
    """Periodic nanoporous film: 100 nm square cell, cylindrical pore of
    porosity 0.25, 200 nm thick, diffuse pore walls and faces."""
    return Workload("pore_film_W100nm_phi0.25_t200nm", material or bvk_holland(),
                    [pore_lattice(100e-9, 0.25, 200e-9, p_pore=p_pore)],
                    SteadyRun(n=n, seed=1005, tally_axis=1, per_bin=True, n_scat_max=10))


def ballistic_transient_e1(n: int = 200_000, nz: int = 30) -> Workload:
    """Ballistic 1-D transient of the paper's Sec. 5.1 (Eq. Analytical_T):
    3 um cube, v = 12360 m/s, tau = 1 s, walls 303 / 297 K at z = 0 / L,
    periodic x, y."""
    mat = Material(omega=np.array([1.0e13]), v=np.array([12360.0]), tau=np.array([1.0]),
                   C=np.array([1.0e6]), T_lin=300.0, name="debye_ballistic")
    g = slab_z(3e-6, 303.0, 297.0, lateral=3e-6)
    t = np.array([5e-12, 50e-12, 100e-12, 200e-12, 300e-12, 900e-12])
    return Workload("ballistic_transient_3um", mat, [g],
                    TransientRun(n=n, seed=7, t_max=float(t[-1]), t_meas=t, grid=(1, 1, nz)))
