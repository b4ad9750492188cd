"""The paper's numerical experiments (Sec. 4) as workloads, run through the C ABI.

* ``shear_thick`` - double shear layer of Sec. 4.1, 1/rho = 15/pi, up to t = 6;
* ``shear_thin``  - thin double shear layer of Sec. 4.2, 1/rho = 50/pi, up to t = 9.5;
* ``kelvin_helmholtz`` - the layer u = (cos y, 0.03 sin(x/2)) of Sec. 4.3 on
  [0, 4pi)^2 up to t = 45 (tau = 0.05, the value of the figure caption; the text says 0).

Each run records, every ``record_every`` steps, the diagnostics the paper plots
(Figs. 2-3: max |D_0 . u| over time) plus the L2 divergence and the enstrophy,
and returns the final vorticity.  The time step follows the workloads' rule
(CFL and viscous bounds) shortened so that the run ends exactly at t_end.

``convergence`` is the study of Tables 1-2 (Sec. 4.1): the thick layer at
eps = 1e-6, tau = 0, WENO3, up to t = 1 on the paper's grids of N = 33, 65,
129, 257 points against its 513 x 513 reference, with the area-weighted L1,
L2 and max norms of the vorticity error and their orders.  The paper does not
say how N counts points on the periodic square; two readings are offered:
"nodes" (N points per side including both ends of the period, so N - 1 cells
and nested grids, compared by injection) and "cells" (N cells, not nested,
the reference evaluated at the coarse cell centres by its trigonometric
interpolant, exact for the band-limited part it resolves).

``uniform_in_eps`` repeats the Table 2 study for several eps at tau = 0 and
0.05 (Fig. 1: the error at fixed N and dt stays bounded as eps varies).

``figures`` runs the flows of Figs. 2-5 of Sec. 4 (thick layer at
eps = 1e-6 with tau = 0 to t = 6 and tau = 0.05 to t = 9.5, the same at
eps = 0.25 (Fig. 3_2, smeared vortices), thin layer at eps = 1e-6 with both
tau), each at the largest of a list of CFL numbers that keeps the run finite
(the inviscid runs need a smaller one), and reports the divergence history,
the enstrophy and the extreme vorticity.

    python -m paper_2512_19847_gb300.experiments --case shear_thin --n 512 --eps 1e-6
    python -m paper_2512_19847_gb300.experiments --table 2
    python -m paper_2512_19847_gb300.experiments --figures
    python -m paper_2512_19847_gb300.experiments --uniform
"""
from __future__ import annotations

import argparse
import json
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import api, tableaux
from . import workloads as W

CASES = {
    "shear_thick": {"init": lambda n: W.double_shear_layer(n, inv_rho=15.0 / math.pi), "L": 2 * math.pi, "t_end": 6.0},
    "shear_thin": {"init": lambda n: W.double_shear_layer(n, inv_rho=50.0 / math.pi), "L": 2 * math.pi, "t_end": 9.5},
    "kelvin_helmholtz": {"init": W.kelvin_helmholtz, "L": 4 * math.pi, "t_end": 45.0},
}


@dataclass
class History:
    case: str
    n: int
    eps: float
    tau: float
    dt: float
    steps: int
    t: list = field(default_factory=list)
    div_max: list = field(default_factory=list)
    div_l2: list = field(default_factory=list)
    enstrophy: list = field(default_factory=list)
    vorticity: torch.Tensor | None = None
    wall_s: float = 0.0

    def summary(self) -> dict:
        return {"case": self.case, "n": self.n, "eps": self.eps, "tau": self.tau, "dt": self.dt, "steps": self.steps,
                "t": self.t, "div_max": self.div_max, "div_l2": self.div_l2, "enstrophy": self.enstrophy,
                "wall_s": round(self.wall_s, 3)}


def run(case: str, n: int, eps: float = 1e-4, tau: float = 0.05, t_end: float | None = None, record_every: int = 50,
        precision: int = api.FP64, scheme: str = "WENO5_C4", mach: float = 1e-2, cfl: float = 0.4,
        visc: float = 0.32) -> History:
    """Run one Sec. 4 experiment on an n x n grid and record its diagnostics
    (cfl, visc: the coefficients of the step's CFL and viscous bounds)."""
    c = CASES[case]
    L = c["L"]
    t_end = c["t_end"] if t_end is None else t_end
    u1, u2, p = c["init"](n)
    dt, steps = W.fixed_time_dt(t_end, W.stable_dt(u1, u2, L / n, tau, cfl=cfl, visc=visc))
    prm = api.default_params(n, n, eps=eps, dt=dt, tau=tau, mach=mach, Lx=L, Ly=L, space_scheme=scheme,
                             tableau=tableaux.gsa2(), precision=precision)
    s = api.Solver(prm)
    s.set_equilibrium(*[torch.from_numpy(a).cuda() for a in (u1, u2, p)])
    h = History(case, n, eps, tau, dt, steps)

    def record(k):
        d = s.diagnostics()
        h.t.append(k * dt)
        h.div_max.append(d["div_max"])
        h.div_l2.append(d["div_l2"])
        h.enstrophy.append(d["enstrophy"])

    t0 = time.perf_counter()
    record(0)
    done = 0
    while done < steps:
        k = min(record_every, steps - done)
        s.step(k)
        done += k
        record(done)
    s.sync_status()
    h.vorticity = s.diagnostics(vorticity=True)["vorticity"]
    h.wall_s = time.perf_counter() - t0
    return h


def _final_vorticity(n: int, tableau, eps: float, tau: float, t_end: float, cfl: float, scheme: str,
                     nodes: bool = False, weno_eps: float = 1e-6) -> np.ndarray:
    u1, u2, p = W.double_shear_layer(n, inv_rho=15.0 / math.pi, nodes=nodes)
    dt, steps = W.fixed_time_dt(t_end, W.cfl_dt(u1, u2, 2 * math.pi / n, cfl))
    prm = api.default_params(n, n, eps=eps, dt=dt, tau=tau, space_scheme=scheme, tableau=tableau, weno_eps=weno_eps)
    s = api.Solver(prm)
    s.set_equilibrium(*[torch.from_numpy(a).cuda() for a in (u1, u2, p)])
    s.step(steps)
    s.sync_status()
    return s.diagnostics(vorticity=True)["vorticity"].cpu().numpy()


def interpolate_periodic(f, n: int):
    """Values at the cell centres of an n x n grid of the trigonometric interpolant
    of f, a cell-centred field of an odd size m on the same periodic square."""
    m = f.shape[0]
    F = np.fft.fft2(f) / (m * m)
    k = np.fft.fftfreq(m, d=1.0 / m)                       # -(m-1)/2 .. (m-1)/2 (m odd: no Nyquist mode)
    s = (np.arange(n) + 0.5) * m / n - 0.5                  # coarse centres in fine index units
    E = np.exp(2j * np.pi * np.outer(s, k) / m)             # n x m
    return np.real(E @ F @ E.T)


def convergence(table: int = 2, sizes=(33, 65, 129, 257), ref: int = 513, eps: float = 1e-6, tau: float = 0.0,
                t_end: float = 1.0, cfl: float = 0.5, scheme: str = "WENO3_C4", grids: str = "nodes",
                weno_eps: float = 1e-6) -> list[dict]:
    """Tables 1-2 of Sec. 4.1: vorticity errors against the finest grid and their orders,
    for the first-order (table 1) or second-order (table 2) GSA IMEX scheme; grids
    "nodes" or "cells" (the two readings of N in the module docstring)."""
    tab = tableaux.euler() if table == 1 else tableaux.gsa2()
    nodes = grids == "nodes"
    cells = (lambda n: n - 1) if nodes else (lambda n: n)
    wref = _final_vorticity(cells(ref), tab, eps, tau, t_end, cfl, scheme, nodes, weno_eps)
    rows, prev = [], None
    for n in sizes:
        w = _final_vorticity(cells(n), tab, eps, tau, t_end, cfl, scheme, nodes, weno_eps)
        if nodes:
            r = cells(ref) // cells(n)
            e = w - wref[::r, ::r]
        else:
            e = w - interpolate_periodic(wref, n)
        h2 = (2 * math.pi / cells(n)) ** 2
        norms = (h2 * np.abs(e).sum(), math.sqrt(h2 * (e * e).sum()), float(np.abs(e).max()))
        orders = [None] * 3 if prev is None else [math.log2(a / b) for a, b in zip(prev, norms)]
        rows.append({"N": n, "L1": norms[0], "L1_order": orders[0], "L2": norms[1], "L2_order": orders[1],
                     "Linf": norms[2], "Linf_order": orders[2]})
        prev = norms
    return rows


def uniform_in_eps(eps_values=(1e-6, 1e-4, 1e-2, 0.25), taus=(0.0, 0.05), sizes=(33, 65, 129), ref: int = 257,
                   cfl: float = 0.5) -> dict:
    """Fig. 1 of Sec. 4.1: the Table 2 study (second-order tableau, WENO3, thick layer,
    t = 1) repeated for several eps at tau = 0 and tau = 0.05; the scheme is uniformly
    accurate in eps when the errors at fixed (N, dt) stay bounded as eps varies."""
    out = {}
    for tau in taus:
        for eps in eps_values:
            out[f"tau{tau:g}_eps{eps:g}"] = convergence(2, sizes=sizes, ref=ref, eps=eps, tau=tau, cfl=cfl)
    return out


FIGURES = {
    "fig2_thick_euler": ("shear_thick", 1e-6, 0.0, 6.0),
    "fig3_thick_ns": ("shear_thick", 1e-6, 0.05, 9.5),
    "fig3_2_thick_euler_eps0.25": ("shear_thick", 0.25, 0.0, 6.0),
    "fig3_2_thick_ns_eps0.25": ("shear_thick", 0.25, 0.05, 9.5),
    "fig4_thin_euler": ("shear_thin", 1e-6, 0.0, 9.5),
    "fig5_thin_ns": ("shear_thin", 1e-6, 0.05, 9.5),
}


def figures(n: int = 256, cfls=(0.4, 0.3, 0.2, 0.1, 0.05), names=None, record_every: int = 25,
            scheme: str = "WENO3_C4") -> dict:
    """The flows of Figs. 2-5 (Sec. 4.1-4.2) on n x n cells with the paper's WENO3
    (Sec. 4.1): for each, the largest CFL number of `cfls` whose run stays finite,
    the divergence history (max |D_0 . u| over time), the enstrophy at the start and
    the end, and the extreme vorticity."""
    out = {}
    for name in names or FIGURES:
        case, eps, tau, t_end = FIGURES[name]
        res = {"case": case, "eps": eps, "tau": tau, "t_end": t_end, "tried": []}
        for cfl in cfls:
            try:
                h = run(case, n, eps=eps, tau=tau, t_end=t_end, record_every=record_every, cfl=cfl, scheme=scheme)
            except api.ApDvmError as e:
                if e.status != 5:            # anything but a non-finite state is an error
                    raise
                res["tried"].append({"cfl": cfl, "finite": False})
                continue
            w = h.vorticity
            res.update({"cfl": cfl, "dt": h.dt, "steps": h.steps, "wall_s": round(h.wall_s, 2),
                        "div_max_final": h.div_max[-1], "div_max_peak": max(h.div_max),
                        "enstrophy_start": h.enstrophy[0], "enstrophy_end": h.enstrophy[-1],
                        "vorticity_max": float(w.abs().max()), "div_history": [h.t[::8], h.div_max[::8]]})
            res["tried"].append({"cfl": cfl, "finite": True})
            break
        out[name] = res
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--case", choices=sorted(CASES), default="shear_thick")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--tau", type=float, default=0.05)
    ap.add_argument("--t-end", type=float, default=None)
    ap.add_argument("--every", type=int, default=50)
    ap.add_argument("--fp32", action="store_true", help="FP32 deviation form")
    ap.add_argument("--cfl", type=float, default=0.4, help="CFL number (0.5 for the convergence study)")
    ap.add_argument("--visc", type=float, default=0.32)
    ap.add_argument("--table", type=int, choices=(1, 2), default=None,
                    help="run the convergence study of Table 1 or 2 instead")
    ap.add_argument("--grids", choices=("nodes", "cells"), default="nodes")
    ap.add_argument("--ref", type=int, default=513, help="reference grid of the convergence study")
    ap.add_argument("--figures", action="store_true", help="run the flows of Figs. 2-5 instead")
    ap.add_argument("--uniform", action="store_true", help="run the eps-uniformity study of Fig. 1 instead")
    args = ap.parse_args()
    if args.table:
        for row in convergence(args.table, grids=args.grids, ref=args.ref, cfl=args.cfl):
            print(json.dumps(row))
        return
    if args.figures:
        print(json.dumps(figures(args.n)))
        return
    if args.uniform:
        print(json.dumps(uniform_in_eps()))
        return
    h = run(args.case, args.n, args.eps, args.tau, args.t_end, args.every,
            api.FP32_DEV if args.fp32 else api.FP64, cfl=args.cfl, visc=args.visc)
    print(json.dumps(h.summary()))


if __name__ == "__main__":
    main()
