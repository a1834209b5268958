"""The five seeded workloads, with their stated seeds and tolerances.

  laplace_n4       vector Laplacian, 4^3 cubes x 6 tets, harmonic quadratic data,
                   plain FP64 AMG-PCG to 1e-10                         (2,187 DOF)
  elasticity_n32   elasticity E=1, nu=0.3, 32^3 cubes, clamped z=0, U[-1,1]^3
                   traction on z=1; FP32 V-cycle in FP64 flexible CG to 1e-8
                                                                       (823,875 DOF)
  stokes_lid_n24   Taylor-Hood Stokes, lid-driven cube 24^3, mean-zero pressure,
                   FP32 inner / FP64 outer flexible GMRES to 1e-8      (368,572 DOF)
  batched_elast    64 box meshes, n ~ U{8..24}, side lengths ~ U[1,4] per axis,
                   nu ~ U[0.2,0.45], 16 N(0,1) traction loads each; SpMM, to 1e-8
  mixed_elast_n40  mixed elasticity, nu in {0.49, 0.499, 0.4999}, 40^3 cubes,
                   vertices jittered by U[-0.2h, 0.2h]; FP32 inner / FP64 outer
                   flexible GMRES(300) to 1e-8 (FGMRES(50) stagnates at nu = 0.4999)
"""
from __future__ import annotations

import numpy as np

from .problems import (elasticity_problem, mixed_elasticity_family, stokes_lid_problem,
                       vector_laplace_problem)

CONFIGS = {
    "laplace_n4": {"tol": 1e-10, "kind": "laplace", "n": 4, "seed": 0},
    "elasticity_n32": {"tol": 1e-8, "kind": "elasticity", "n": 32, "seed": 1},
    "stokes_lid_n24": {"tol": 1e-8, "kind": "stokes", "n": 24},
    "batched_elast": {"tol": 1e-8, "kind": "elasticity", "n_problems": 64, "n_rhs": 16,
                      "seed": 4},
    "mixed_elast_n40": {"tol": 1e-8, "kind": "mixed", "n": 40, "nus": (0.49, 0.499, 0.4999),
                        "seed": 5, "gmres_restart": 300},
}


def batched_specs(n_problems: int = 64, seed: int = 4, n_range=(8, 24)):
    """Per-problem (n, lengths, nu, seed) of the batched workload, drawn in order."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n_problems):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        lengths = tuple(float(v) for v in rng.uniform(1.0, 4.0, size=3))
        nu = float(rng.uniform(0.2, 0.45))
        specs.append({"n": n, "lengths": lengths, "nu": nu, "seed": 10_000 + i})
    return specs


def make_config(name: str, n: int | None = None, **over):
    """Build the problem(s) of a named workload; `n` overrides the mesh size."""
    cfg = dict(CONFIGS[name])
    cfg.update(over)
    if n is not None:
        cfg["n"] = n
    if name.startswith("laplace"):
        return vector_laplace_problem(cfg["n"], seed=cfg["seed"])
    if name.startswith("elasticity"):
        return elasticity_problem(cfg["n"], seed=cfg["seed"], E=1.0, nu=0.3)
    if name.startswith("stokes"):
        return stokes_lid_problem(cfg["n"])
    if name.startswith("mixed"):
        return mixed_elasticity_family(cfg["n"], cfg["nus"], seed=cfg["seed"])
    if name.startswith("batched"):
        return [elasticity_problem(s["n"], seed=s["seed"], nu=s["nu"], lengths=s["lengths"],
                                   n_rhs=cfg["n_rhs"], traction="gaussian")
                for s in batched_specs(cfg["n_problems"], cfg["seed"])]
    raise KeyError(name)
