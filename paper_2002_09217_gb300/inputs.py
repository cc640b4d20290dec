"""Seeded synthetic inputs for the PonD step: initial (rho, u, T) fields and
workload parameters.

This module generates data only (profiles, counter-based noise, request mixes);
it holds none of the method's arithmetic, and both the CUDA path and the test
oracle consume what it returns.  Thermodynamic constants (Maxwell coexistence
densities, Rankine-Hugoniot post-shock states, the per-temperature time step)
are read from ``workloads.json`` next to this file.

Noise: rho <- rho (1 + xi), xi ~ U[-A, A] drawn from splitmix64(seed ^ node).
"""
from __future__ import annotations

import dataclasses
import functools
import json
import math
import os

import numpy as np

SEED = 20020921
A_VDW, B_VDW, R_GAS = 2.0 / 49.0, 2.0 / 21.0, 1.0
_HERE = os.path.dirname(os.path.abspath(__file__))


@functools.lru_cache(maxsize=1)
def table() -> dict:
    with open(os.path.join(_HERE, "workloads.json")) as fh:
        return json.load(fh)


def t_cr() -> float:
    return table()["critical"]["T"]


def coexistence(Tr: float) -> tuple[float, float, float]:
    """(rho_v, rho_l, dt) at the tabulated reduced temperature nearest to Tr."""
    row = table()["coexistence"]["%.2f" % round(Tr, 2)]
    return row["rho_v"], row["rho_l"], row["dt"]


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """n uniforms in [0, 1) from splitmix64(seed ^ k), k = 0..n-1 (counter based)."""
    with np.errstate(over="ignore"):
        z = (np.arange(n, dtype=np.uint64) ^ np.uint64(seed)) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def noise(seed: int, shape, amp: float) -> np.ndarray:
    n = int(np.prod(shape))
    return (2.0 * splitmix64_uniform(seed, n) - 1.0).reshape(shape) * amp


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    bc_x: int
    bc_y: int
    T_r: float
    kappa: float
    tau: float
    dt: float
    steps: int
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    T: np.ndarray
    a: float = A_VDW
    b: float = B_VDW
    R: float = R_GAS
    delta: float = 1.0 / 3.0
    k_cond: float = -1.0
    p_floor: float = 0.05 / 6.0     # 5 % of p_cr
    eos: str = "vdw"                # or "dieterici" / "simplified" (isothermal)
    isothermal: bool = False        # T held at its (uniform) initial value
    eos_params: tuple = ()          # (beta, rho_l, rho_v, p0) of "simplified"

    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    def fields(self):
        return self.rho, self.ux, self.uy, self.T


def slab(nx=128, ny=4, Tr=0.9, width=4.0, amp=1e-3, steps=2000, seed=SEED, kappa=0.02, tau=1.0):
    """Liquid slab over the middle half of a periodic box, vapour elsewhere."""
    rv, rl, dt = coexistence(Tr)
    x = np.arange(nx) + 0.5
    prof = rv + (rl - rv) * 0.5 * (np.tanh((x - nx / 4) / width) - np.tanh((x - 3 * nx / 4) / width))
    rho = np.tile(prof, (ny, 1)) * (1.0 + noise(seed, (ny, nx), amp))
    z = np.zeros((ny, nx))
    return Workload("slab%dx%d" % (nx, ny), nx, ny, 0, 0, Tr, kappa, tau, dt, steps, rho, z, z.copy(),
                    np.full((ny, nx), Tr * t_cr()))


def shock_tube(nx=2048, ny=4, Tr=1.1, rho_left=7.0, rho_right=1.75, width=4.0, steps=5000,
               tau=1.0):
    """Supercritical two-state tube, smooth tanh step at the middle, zero-gradient
    ends in x, periodic in y."""
    x = np.arange(nx) + 0.5
    prof = rho_right + (rho_left - rho_right) * 0.5 * (1.0 - np.tanh((x - nx / 2) / width))
    rho = np.tile(prof, (ny, 1))
    z = np.zeros((ny, nx))
    dt = table()["supercritical_1.10"]["dt"] if abs(Tr - 1.1) < 1e-12 else 0.4
    return Workload("shocktube%dx%d" % (nx, ny), nx, ny, 1, 0, Tr, 0.0, tau, dt, steps, rho, z,
                    z.copy(), np.full((ny, nx), Tr * t_cr()))


def droplet(n=512, Tr=0.85, radius=64.0, width=4.0, amp=1e-4, steps=20000, seed=SEED, kappa=0.02,
            tau=1.0, ny=None):
    """Liquid disc at the box centre in its vapour, periodic."""
    ny = n if ny is None else ny
    rv, rl, dt = coexistence(Tr)
    x = np.arange(n)[None, :] + 0.5
    y = np.arange(ny)[:, None] + 0.5
    r = np.sqrt((x - n / 2) ** 2 + (y - ny / 2) ** 2)
    rho = (rv + (rl - rv) * 0.5 * (1.0 - np.tanh((r - radius) / width))) * (1.0 + noise(seed, (ny, n), amp))
    z = np.zeros((ny, n))
    return Workload("droplet%dx%d" % (n, ny), n, ny, 0, 0, Tr, kappa, tau, dt, steps, rho, z,
                    z.copy(), np.full((ny, n), Tr * t_cr()))


@dataclasses.dataclass
class Workload3:
    """A three-dimensional (D3Q27) workload: fields of shape (nz, ny, nx)."""
    name: str
    nx: int
    ny: int
    nz: int
    bc_x: int
    bc_y: int
    bc_z: int
    T_r: float
    kappa: float
    tau: float
    dt: float
    steps: int
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    uz: np.ndarray
    T: np.ndarray
    a: float = A_VDW
    b: float = B_VDW
    R: float = R_GAS
    delta: float = 1.0 / 3.0
    k_cond: float = -1.0
    p_floor: float = 0.05 / 6.0

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz

    def fields(self):
        return self.rho, self.ux, self.uy, self.uz, self.T


def droplet3d(n=96, Tr=0.85, radius=20.0, width=4.0, amp=1e-4, steps=2000, seed=SEED, kappa=0.02,
              tau=1.0, ny=None, nz=None, bc_z=0):
    """Liquid sphere at the box centre in its vapour (D3Q27), periodic in x and y."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    rv, rl, dt = coexistence(Tr)
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(n) + 0.5, indexing="ij")
    r = np.sqrt((x - n / 2) ** 2 + (y - ny / 2) ** 2 + (z - nz / 2) ** 2)
    rho = (rv + (rl - rv) * 0.5 * (1.0 - np.tanh((r - radius) / width))) * (1.0 + noise(seed, (nz, ny, n), amp))
    zero = np.zeros((nz, ny, n))
    return Workload3("droplet3d%dx%dx%d" % (n, ny, nz), n, ny, nz, 0, 0, bc_z, Tr, kappa, tau, dt, steps,
                     rho, zero, zero.copy(), zero.copy(), np.full((nz, ny, n), Tr * t_cr()))


def from_workload3(w, precision="mixed", **kw):
    """Keyword arguments of a D3Q27 ``pond.Simulation`` for a ``Workload3``."""
    d = dict(bc_x=w.bc_x, bc_y=w.bc_y, bc_z=w.bc_z, nz=w.nz, a=w.a, b=w.b, R=w.R, delta=w.delta,
             kappa=w.kappa, tau=w.tau, precision=precision, dt=w.dt, k_cond=w.k_cond, p_floor=w.p_floor,
             lattice="d3q27")
    d.update(kw)
    return d


def coexistence_slab(Tr=0.9, delta=1.0 / 3.0, advected=False, nx=256, ny=1, width=4.0, steps=8000,
                     kappa=0.02, tau=1.0):
    """A liquid slab over the middle half of a periodic box in its vapour at the Maxwell
    densities, T uniform: the coexistence curve of the main text's Fig. 2 for delta = 1/3
    or 2/3, and for delta = 1/3 advected with the uniform velocity U = 5 U_ch
    (``advected=True``).  The time step comes from the workload table for each case."""
    rv, rl, dt = coexistence(Tr)
    fig = table()["figure2"]
    key = "%.2f" % round(Tr, 2)
    U = 0.0
    if advected:
        if abs(delta - 1.0 / 3.0) > 1e-12:
            raise ValueError("the advected case is tabulated for delta = 1/3")
        U, dt = fig["U"], fig["dt_advected"][key]
        tag = "adv"
    elif abs(delta - 2.0 / 3.0) < 1e-12:
        dt = fig["dt_delta_2_3"][key]
        tag = "d23"
    elif abs(delta - 1.0 / 3.0) < 1e-12:
        tag = "d13"
    else:
        raise ValueError("delta must be 1/3 or 2/3")
    x = np.arange(nx) + 0.5
    prof = rv + (rl - rv) * 0.5 * (np.tanh((x - nx / 4) / width) - np.tanh((x - 3 * nx / 4) / width))
    rho = np.tile(prof, (ny, 1))
    z = np.zeros((ny, nx))
    return Workload("coex%s%.2f_%dx%d" % (tag, Tr, nx, ny), nx, ny, 0, 0, Tr, kappa, tau, dt, steps, rho,
                    z + U, z.copy(), np.full((ny, nx), Tr * t_cr()), delta=delta)


def dieterici_slab(Tr=0.9, nx=256, ny=1, width=4.0, steps=None, kappa=0.02, tau=1.0):
    """Isothermal coexistence with the Dieterici EoS (SM "Coexistence curve"): a liquid
    slab over the middle half of a periodic box in its vapour at the Maxwell densities of
    that EoS, T held at Tr T_cr; p_floor at 5 % of its p_cr (never reached: the Dieterici
    pressure is positive).  Default steps: a relaxation time of 1500."""
    d = table()["dieterici"]
    row = d["coexistence"]["%.2f" % round(Tr, 2)]
    rv, rl, dt = row["rho_v"], row["rho_l"], row["dt"]
    steps = int(math.ceil(1500.0 / dt)) if steps is None else steps
    x = np.arange(nx) + 0.5
    prof = rv + (rl - rv) * 0.5 * (np.tanh((x - nx / 4) / width) - np.tanh((x - 3 * nx / 4) / width))
    rho = np.tile(prof, (ny, 1))
    z = np.zeros((ny, nx))
    return Workload("dieterici%.2f_%dx%d" % (Tr, nx, ny), nx, ny, 0, 0, Tr, kappa, tau, dt, steps, rho,
                    z, z.copy(), np.full((ny, nx), Tr * d["critical"]["T"]), a=d["a"], b=d["b"],
                    p_floor=0.05 * d["critical"]["p"], eos="dieterici", isothermal=True)


def nonclassical_tube(case="fig4", nx=1024, ny=1, width=2.0, tau=1.0):
    """Shock tubes of non-classical gas dynamics in the van der Waals fluid: the anomalous
    case of the main text's Fig. 4 (delta = 0.0125, both states with Gamma < 0) and the
    SM's cases "I" (delta = 0.329, classical) and "II" (delta = 0.0125, Gamma changes sign
    during the flow).  Left / right states at rest from the workload table, a tanh step of
    `width` nodes at the middle, zero-gradient ends in x, periodic in y, kappa = 0; steps
    up to the case's snapshot time t* = (t / nx) sqrt(p_cr / rho_cr)."""
    tab = table()["nonclassical"]
    c = tab["cases"][case]
    x = np.arange(nx) + 0.5
    sw = 0.5 * (1.0 - np.tanh((x - nx / 2) / width))
    rho = np.tile(c["right"]["rho"] + (c["left"]["rho"] - c["right"]["rho"]) * sw, (ny, 1))
    T = np.tile(c["right"]["T"] + (c["left"]["T"] - c["right"]["T"]) * sw, (ny, 1))
    z = np.zeros((ny, nx))
    steps = int(round(c["t_star"] * nx / tab["U_ch"] / c["dt"]))
    return Workload("nonclassical_%s_%dx%d" % (case, nx, ny), nx, ny, 1, 0, 1.0, 0.0, tau, c["dt"],
                    steps, rho, z, z.copy(), T, delta=c["delta"])


def simplified_eos(kind="slab", phase="liquid", nx=256, ny=1, width=4.0, amp=1e-3, pulse_width=12.0,
                   steps=None, kappa=0.1, tau=1.0):
    """The SM's simplified near-critical EoS (double-well free energy, density ratio 10),
    isothermal: kind "slab" is a liquid slab over the middle half of a periodic box in its
    vapour at the two saturated densities; kind "pulse" a uniform saturated `phase` with
    a Gaussian density bump of relative amplitude `amp` at x = nx/4 (kappa = 0).  T is a
    placeholder (the EoS does not depend on it).  The slab takes dt <= 0.1: across its
    interface the gauge temperature changes tenfold through the double well's spinodal,
    and dt = 0.25 diverged there (the bulk-state rule gives 0.5)."""
    sp = table()["simplified"]
    rl, rv, dt = sp["rho_l"], sp["rho_v"], sp["dt"]
    x = np.arange(nx) + 0.5
    if kind == "slab":
        prof = rv + (rl - rv) * 0.5 * (np.tanh((x - nx / 4) / width) - np.tanh((x - 3 * nx / 4) / width))
        dt = min(dt, 0.1)
        steps = int(math.ceil(1500.0 / dt)) if steps is None else steps
        name = "simplified_slab_%dx%d" % (nx, ny)
    elif kind == "pulse":
        rho0 = rl if phase == "liquid" else rv
        prof = rho0 * (1.0 + amp * np.exp(-((x - 0.0 - nx / 4) / pulse_width) ** 2))
        kappa = 0.0
        steps = 40000 if steps is None else steps
        name = "simplified_%s_pulse_%dx%d" % (phase, nx, ny)
    else:
        raise ValueError("kind must be slab or pulse")
    rho = np.tile(prof, (ny, 1))
    z = np.zeros((ny, nx))
    return Workload(name, nx, ny, 0, 0, 1.0, kappa, tau, dt, steps, rho, z, z.copy(), np.full((ny, nx), 0.1),
                    p_floor=1e-4, eos="simplified", isothermal=True,
                    eos_params=(sp["beta"], rl, rv, sp["p0"]))


def sound_pulse(Tr=0.9, phase="vapour", nx=2048, ny=1, amp=1e-3, width=12.0, steps=40000, tau=1.0,
                isothermal=False):
    """Uniform saturated vapour or liquid at T = Tr T_cr (phase "vapour" / "liquid"), or
    the critical state (phase "critical"), periodic and at rest, with a Gaussian density
    bump of relative amplitude `amp` and width `width` nodes at x = nx/4 and the
    temperature left uniform: the bump splits into two sound pulses and a standing
    entropy mode (the speed-of-sound benchmark of the main text, Fig. 1).  kappa = 0: a
    single phase has no interface.  isothermal=True holds T (the SM's isothermal speed of
    sound)."""
    tab = table()
    if phase == "critical":
        rho0, T0, dt = tab["critical"]["rho"], tab["critical"]["T"], tab["sound"]["critical"]["dt"]
        Tr = 1.0
        name = "soundcrit%dx%d" % (nx, ny)
    elif phase in ("vapour", "liquid"):
        rv, rl, _ = coexistence(Tr)
        row = tab["sound"]["%.2f" % round(Tr, 2)]
        rho0, dt = (rv, row["dt_v"]) if phase == "vapour" else (rl, row["dt_l"])
        T0 = Tr * t_cr()
        name = "sound%s%.2f_%dx%d" % (phase[0], Tr, nx, ny)
    else:
        raise ValueError("phase must be vapour, liquid or critical")
    x = np.arange(nx) + 0.0
    prof = rho0 * (1.0 + amp * np.exp(-((x - nx / 4) / width) ** 2))
    rho = np.tile(prof, (ny, 1))
    z = np.zeros((ny, nx))
    return Workload(name + ("_iso" if isothermal else ""), nx, ny, 0, 0, Tr, 0.0, tau, dt, steps, rho, z,
                    z.copy(), np.full((ny, nx), T0), isothermal=isothermal)


def droplet_shock(nx=2048, ny=1024, Tr=0.8, radius=80.0, xc=600.0, x_shock=300.0, Mach=1.5,
                  width=4.0, steps=10000, kappa=0.02, tau=1.0):
    """Droplet at coexistence in its vapour, hit by a planar shock (post-shock state
    on the left of x_shock); zero-gradient boundaries."""
    rv, rl, dt = coexistence(Tr)
    sh = table()["shock"]["%.2f" % round(Tr, 2)]["%.1f" % round(Mach, 1)]
    Tc = t_cr()
    x = np.arange(nx)[None, :] + 0.5 + np.zeros((ny, 1))
    y = np.arange(ny)[:, None] + 0.5 + np.zeros((1, nx))
    r = np.sqrt((x - xc) ** 2 + (y - ny / 2) ** 2)
    drop = 0.5 * (1.0 - np.tanh((r - radius) / width))
    post = 0.5 * (1.0 - np.tanh((x - x_shock) / width))
    rho = rv + (rl - rv) * drop + (sh["rho1"] - rv) * post
    ux = sh["u1"] * post
    T = Tr * Tc + (sh["T1"] - Tr * Tc) * post
    return Workload("dropletshock%dx%d" % (nx, ny), nx, ny, 1, 1, Tr, kappa, tau, sh["dt_droplet"], steps,
                    rho, ux, np.zeros((ny, nx)), T)


def shock_in_vapour(n=64, Tr=0.8, Mach=1.5, width=4.0, steps=1000, kappa=0.02, tau=1.0):
    """Square box of vapour at coexistence density with a planar shock entering from
    the left (zero-gradient in x, periodic in y)."""
    rv, rl, dt = coexistence(Tr)
    sh = table()["shock"]["%.2f" % round(Tr, 2)]["%.1f" % round(Mach, 1)]
    Tc = t_cr()
    x = np.arange(n)[None, :] + 0.5 + np.zeros((n, 1))
    post = 0.5 * (1.0 - np.tanh((x - n / 4) / width))
    rho = rv + (sh["rho1"] - rv) * post
    return Workload("shock%d" % n, n, n, 1, 0, Tr, kappa, tau, sh["dt"], steps, rho, sh["u1"] * post,
                    np.zeros((n, n)), Tr * Tc + (sh["T1"] - Tr * Tc) * post)


CONFIGS = {
    "slab128x4": lambda: slab(),
    "shocktube2048x4": lambda: shock_tube(),
    "droplet512x512": lambda: droplet(),
    "dropletshock2048x1024": lambda: droplet_shock(),
}


def config(name: str) -> Workload:
    return CONFIGS[name]()


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float
    side: int
    T_r: float
    kind: str
    mach: float
    steps: int
    precision: str


def serving_requests(n: int = 256, rate: float = 1.0, seed: int = SEED) -> list[Request]:
    """Seeded request mix: Poisson arrivals at the given rate (per second), square
    sides log-uniform in [64, 1024], T/T_cr uniform in [0.70, 0.95] (tabulated to
    0.01), init in {droplet, slab, shock}, shock Mach uniform in [1.2, 3.0]
    (tabulated to 0.1), 1000-10000 steps, precision mixed or fp64 (50/50)."""
    u = splitmix64_uniform(seed ^ 0x5EEDF00D, 8 * n).reshape(n, 8)
    reqs = []
    t = 0.0
    for k in range(n):
        t += -math.log(1.0 - u[k, 0]) / rate
        side = int(round(math.exp(math.log(64) + u[k, 1] * (math.log(1024) - math.log(64)))))
        Tr = round(0.70 + 0.25 * u[k, 2], 2)
        kind = ("droplet", "slab", "shock")[min(2, int(u[k, 3] * 3))]
        mach = round(1.2 + 1.8 * u[k, 4], 1)
        steps = 1000 + int(u[k, 5] * 9001)
        prec = "mixed" if u[k, 6] < 0.5 else "fp64"
        reqs.append(Request(k, t, side, Tr, kind, mach, min(steps, 10000), prec))
    return reqs


def request_workload(req: Request) -> Workload:
    n = req.side
    if req.kind == "droplet":
        return droplet(n=n, Tr=req.T_r, radius=n / 8.0, steps=req.steps, seed=SEED + req.rid)
    if req.kind == "slab":
        return slab(nx=n, ny=n, Tr=req.T_r, steps=req.steps, seed=SEED + req.rid)
    return shock_in_vapour(n=n, Tr=req.T_r, Mach=req.mach, steps=req.steps)
