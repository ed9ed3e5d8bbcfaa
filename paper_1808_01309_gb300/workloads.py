"""Named workloads: the configurations this library is measured and tested on,
as plan keyword arguments plus their seeded initial state and forcing.

Host-side recipes only (they hold no step of the method):

  taylor_green_32    32^3 FP64 Taylor-Green vortex, nu = 1e-2, dt = 1e-3,
                     IF-RK2, 10 steps, unforced
  forced_<n>         n^3 forced hydrodynamics: seeded solenoidal field with
                     E(K) ~ K^4 exp(-2 (K/4)^2), E = 0.5 (seed 1), forcing on
                     shells 2 <= |k| <= 3 (seed 2), nu = 2e-3, dt = 1e-3,
                     IF-RK4 (n = 256: 100 steps, FP32 and FP64; 512, 1024:
                     10 steps, FP32)
  mhd_512            u as forced_512, B from the same spectrum (seed 51),
                     eta = nu
  boussinesq_512     u as forced_512, theta from the same spectrum shape
                     (seed 61, variance 0.5), N = 1, kappa = nu
  ensemble_48        48 unforced members, 16 each at 64^3, 96^3, 128^3,
                     seeds 1000 + i, nu_i = 1e-3 + 4e-3 U(seed 2000 + i),
                     FP32, IF-RK4, dt = 1e-3, 50 steps

Usage:
    w = workloads.get("forced_512")
    plan = ps.Plan(*w.shape, **w.plan_kwargs(forcing=torch_forcing))
    u0 = w.initial_state()          # numpy complex128, state layout
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import inputs


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    shape: tuple            # (nx, ny, nz)
    prec: str               # "fp32" or "fp64"
    eq: str = "hd"          # "hd", "mhd", "boussinesq"
    nu: float = 0.0
    eta: float = 0.0
    n_bv: float = 0.0
    kappa: float = 0.0
    rk_order: int = 4
    dt: float = 1e-3
    steps: int = 10
    init: str = "random"    # "random" or "taylor_green"
    seed: int = 1
    forcing_seed: int | None = None

    def plan_kwargs(self, forcing=None) -> dict:
        """Keyword arguments of ps.Plan / ps.make_config (without the grid)."""
        from . import ps
        return dict(prec=ps.Precision.FP32 if self.prec == "fp32" else ps.Precision.FP64,
                    eq={"hd": ps.Equations.HD, "mhd": ps.Equations.MHD,
                        "boussinesq": ps.Equations.BOUSSINESQ}[self.eq],
                    nu=self.nu, eta=self.eta, n_bv=self.n_bv, kappa=self.kappa,
                    rk_order=self.rk_order, forcing=forcing)

    def initial_state(self) -> np.ndarray:
        nx, ny, nz = self.shape
        if self.init == "taylor_green":
            u = inputs.taylor_green(nx, ny, nz)
        else:
            u = inputs.random_solenoidal_field(nx, ny, nz, seed=self.seed)
        if self.eq == "mhd":
            return np.concatenate([u, inputs.random_solenoidal_field(nx, ny, nz, seed=51)])
        if self.eq == "boussinesq":
            return np.concatenate([u, inputs.random_scalar_field(nx, ny, nz, seed=61)])
        return u

    def forcing(self):
        """Velocity forcing in the state layout (three components), or None."""
        if self.forcing_seed is None:
            return None
        nx, ny, nz = self.shape
        return inputs.forcing_field(nx, ny, nz, seed=self.forcing_seed)


def forced(n: int, prec: str = "fp32", steps: int = 10) -> Workload:
    return Workload(f"forced_{n}" + ("" if prec == "fp32" else "_fp64"), (n, n, n), prec, nu=2e-3,
                    steps=steps, seed=1, forcing_seed=2)


ENSEMBLE_SIZES = [64] * 16 + [96] * 16 + [128] * 16


def ensemble_48() -> list:
    """The 48 members of the batched-ensemble workload (unforced)."""
    return [Workload(f"ensemble_48[{i}]", (n, n, n), "fp32", nu=inputs.ensemble_viscosity(i), steps=50,
                     seed=1000 + i) for i, n in enumerate(ENSEMBLE_SIZES)]


_NAMED = {
    "taylor_green_32": lambda: Workload("taylor_green_32", (32, 32, 32), "fp64", nu=1e-2, rk_order=2,
                                        steps=10, init="taylor_green"),
    "forced_256": lambda: forced(256, "fp32", 100),
    "forced_256_fp64": lambda: forced(256, "fp64", 100),
    "forced_512": lambda: forced(512),
    "forced_1024": lambda: forced(1024),
    "mhd_512": lambda: dataclasses.replace(forced(512), name="mhd_512", eq="mhd", eta=2e-3),
    "boussinesq_512": lambda: dataclasses.replace(forced(512), name="boussinesq_512", eq="boussinesq",
                                                  n_bv=1.0, kappa=2e-3),
}


def names() -> list:
    return sorted(_NAMED) + ["ensemble_48"]


def get(name: str):
    """A named workload (a list of members for "ensemble_48")."""
    if name == "ensemble_48":
        return ensemble_48()
    if name not in _NAMED:
        raise KeyError(f"unknown workload {name!r}; known: {', '.join(names())}")
    return _NAMED[name]()
